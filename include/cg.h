/*
 * cg.h -- C ABI of libcg, GPU transfer checks in the manner of Cudagrind
 * (Baumann & Gracia, "Cudagrind: A Valgrind Extension for CUDA", 2013).
 *
 * Cudagrind wraps the CUDA driver calls that allocate, free and copy device
 * memory.  It keeps a list of live device allocations (paper, Fig. 2 caption)
 * and checks every copy against that list and against Memcheck's shadow of
 * host memory (Sec. 2 itemize): copies into or out of unallocated device
 * memory, undefined host data copied to the device, copies larger than their
 * allocation.  Definedness then travels with the data in all three directions
 * (Sec. 5).  libcg runs those checks on the GPU.
 *
 * Model
 *  - Device addresses are plain 64-bit integers (the caller's pointers); libcg
 *    never touches the memory they name.  It keeps, per live allocation, a
 *    device-resident V shadow (1 byte per device byte, bit set = undefined),
 *    all 0xFF when the allocation is registered.
 *  - The host shadow image is caller-owned DEVICE memory (e.g. a torch
 *    tensor) bound with cg_bind_host_shadow: a packed A bitmap (host byte p
 *    <-> bit p&7 of a_bits[p>>3], 1 = addressable) and a V mask (1 byte per
 *    host byte, bit set = undefined).  "Host addresses" in requests are byte
 *    offsets into this image.
 *  - Per byte of a copy: UNADDR if its host byte is unaddressable; else UNDEF
 *    if its V mask is nonzero; else GOOD.  Unaddressable takes precedence.
 *
 * Conventions
 *  - Every function returns cg_status: CG_OK (0) or a negative API error.
 *    Check verdicts are never status codes; they live in cg_report.
 *  - `stream` arguments are cudaStream_t values passed as void* (NULL = the
 *    legacy default stream).  libcg enqueues its work there.
 *  - One cg_ctx must not be used from two host threads at once.
 *  - Pointers documented "device" must be device-accessible memory of the
 *    current device; "host" pointers are ordinary host memory.
 */
#ifndef CG_H
#define CG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------- constants */

typedef int32_t cg_status;
#define CG_OK 0
#define CG_E_ARG -1         /* null pointer or bad argument */
#define CG_E_KIND -2        /* copy kind not HTOD/DTOH/DTOD */
#define CG_E_HOST_RANGE -3  /* host range outside the bound host image */
#define CG_E_ZERO_SIZE -4   /* registering a zero-size allocation */
#define CG_E_WRAP -5        /* allocation range wraps 2^64 */
#define CG_E_OVERLAP -6     /* allocation overlaps a live one; table unchanged */
#define CG_E_NOMEM -7       /* device or host memory for the shadow ran out */
#define CG_E_RANGE -8       /* mark/read range not inside one live allocation */
#define CG_E_CUDA -9        /* a CUDA runtime call failed (see cg_last_error) */
#define CG_E_NO_HOST -10    /* no host shadow image bound */
#define CG_E_ALIGN -11      /* pointer or size breaks an alignment rule */
#define CG_E_STATE -12      /* call not allowed in the context's state */
#define CG_E_TIMEOUT -13    /* a bounded wait ran out */
#define CG_E_FULL -14       /* a queue or ring is full */
#define CG_E_TOO_BIG -15    /* size above a documented maximum */

/* copy kinds (Sec. 5: host/device, device/host, device/device) */
#define CG_HTOD 1u
#define CG_DTOH 2u
#define CG_DTOD 3u

/* per-byte classes, cg_report.first_bad_kind */
#define CG_BYTE_GOOD 0u
#define CG_BYTE_UNADDR 1u
#define CG_BYTE_UNDEF 2u

/* cg_report.flags; cg_err_record.cls is the bit index */
#define CG_F_UNALLOC_DST (1u << 0)   /* dst pointer in no live allocation */
#define CG_F_UNALLOC_SRC (1u << 1)   /* src pointer in no live allocation */
#define CG_F_OVERRUN_DST (1u << 2)   /* dst range runs past its allocation */
#define CG_F_OVERRUN_SRC (1u << 3)   /* src range runs past its allocation */
#define CG_F_HOST_UNADDR (1u << 4)   /* host bytes not addressable */
#define CG_F_HOST_UNDEF (1u << 5)    /* HtoD: undefined host bytes sent */
#define CG_F_DEV_UNDEF_SRC (1u << 6) /* DtoH/DtoD: undefined device bytes (warning) */
#define CG_F_DTOD_OVERLAP (1u << 7)  /* DtoD src and dst overlap (warning) */
#define CG_F_CONCURRENT (1u << 8)    /* served: races a copy of another client (warning) */
#define CG_NFLAGS 9
/* Not a finding: set when a kernel's bounded wait for its own data ran out;
 * the counts of such a report are not valid (cg_check_copy then returns
 * CG_E_TIMEOUT).  Never produces a record. */
#define CG_F_INCOMPLETE (1u << 31)

/* cg_free verdicts */
#define CG_FREE_OK 0u
#define CG_FREE_UNKNOWN 1u  /* no allocation ever had this base */
#define CG_FREE_DOUBLE 2u   /* base of an allocation already freed */
#define CG_FREE_INTERIOR 3u /* inside a live allocation, not its base */

/* ----------------------------------------------------------------- types */

/* One copy to check.  kind selects which fields are host offsets:
 *   CG_HTOD: dst = device address, src = host offset
 *   CG_DTOH: dst = host offset,    src = device address
 *   CG_DTOD: dst = device address, src = device address
 * reserved must be 0.  32 bytes. */
typedef struct cg_copy {
  uint32_t kind;
  uint32_t reserved;
  uint64_t dst;
  uint64_t src;
  uint64_t n;
} cg_copy;

/* The verdict of one copy check (Sec. 2 itemize; Listing 5's expected and
 * found bytes).  Offsets are relative to the copy start; -1 = none.
 * found_x = bytes from the x pointer to the end of the allocation holding
 * it (0 when none does, or when x is the host side).  alloc_*_x describe
 * that allocation.  n_good + n_unaddr + n_undef == expected == n. */
typedef struct cg_report {
  uint32_t flags;
  uint32_t first_bad_kind;
  int64_t first_bad_off;
  int64_t first_unaddr_off;
  int64_t first_undef_off;
  uint64_t n_good;
  uint64_t n_unaddr;
  uint64_t n_undef;
  uint64_t expected;
  uint64_t found_dst;
  uint64_t found_src;
  uint64_t alloc_base_dst;
  uint64_t alloc_size_dst;
  uint64_t alloc_base_src;
  uint64_t alloc_size_src;
  int64_t race_seq; /* CONCURRENT: seq of the copy it races with, else -1 */
} cg_report; /* 120 bytes */

/* One error or warning, emitted per set report flag in (req, cls) order.
 *   UNALLOC_*:     off 0,            count n,             found 0
 *   OVERRUN_*:     off found,        count n - found,     found = found
 *   HOST_UNADDR:   off first unaddr, count n_unaddr,      found n - n_unaddr
 *   HOST_UNDEF / DEV_UNDEF_SRC: off first undef, count n_undef, found n_good
 *   DTOD_OVERLAP:  off dst - src,    count overlap bytes, found 0
 *   CONCURRENT:    off race_seq,     count n,             found 0
 * severity: 0 error, 1 warning (DEV_UNDEF_SRC unless strict; DTOD_OVERLAP;
 * CONCURRENT). */
typedef struct cg_err_record {
  uint64_t req;
  uint32_t cls;
  uint32_t severity;
  int64_t off;
  uint64_t count;
  uint64_t expected;
  uint64_t found;
} cg_err_record; /* 48 bytes */

typedef struct cg_config {
  uint32_t carry;               /* 1 (default): V shadow travels with copies */
  uint32_t strict_device_undef; /* 1: undefined device-source bytes are errors */
  uint64_t shadow_slab_bytes;   /* device shadow pool slab; 0 = 1 GiB */
  uint64_t shadow_budget_bytes; /* cap on the device shadow pool; 0 = none */
  uint32_t scan_ctas_per_sm;    /* single-check grid; 0 = automatic */
  uint32_t batch_segment_kib;   /* batched work split, rounded up to whole
                                   engine steps (4 KiB TMA, 2 KiB registers);
                                   0 = chosen per batch (cg_choose_segment) */
  uint32_t batch_ctas_per_sm;   /* batched grid; 0 = automatic */
  uint32_t scan_engine;         /* scan loads, single and batched checks:
                                   0 auto (= 2), 1 registers, 2 TMA bulk copies */
  uint32_t batch_autotune;      /* 1: with batch_segment_kib = 0, batches of a
                                   new shape first try the split candidates
                                   16..256 KiB in turn (real runs, timed), then
                                   keep the fastest (see cg_choose_segment) */
  uint32_t batch_direct_launch; /* 1: issue a batch's kernels one by one;
                                   0 (default): capture them into a CUDA graph
                                   (updated in place when the next batch has
                                   the same shape) and launch that */
  uint32_t batch_piece_kib;     /* batches on the TMA engine: a host->device
                                   copy that carries nothing and is longer than
                                   1.5x this is planned in pieces of about this
                                   size (whole tiles), each ordered only after
                                   the writes it overlaps; 0 = 1024 (1 MiB),
                                   0xFFFFFFFF = whole copies only */
  uint32_t reserved[5];
} cg_config;

typedef struct cg_ctx cg_ctx;

typedef struct cg_stats {
  uint64_t checks;        /* copies checked (single + batched) */
  uint64_t bytes_checked; /* sum of n */
  uint64_t batches;
  uint64_t levels;        /* dependency levels run by batches */
  uint64_t kernels;       /* kernels launched by this context */
  uint64_t errors[CG_NFLAGS]; /* reports per flag */
  uint64_t live_allocs;
  uint64_t shadow_bytes;  /* device shadow pool held */
  uint64_t batch_ns;      /* wall time inside cg_check_batch */
  uint64_t batch_plan_ns; /* of which: host dependency planning */
  uint64_t batch_lookup_ns; /* of which: device lookup incl. its read-back */
  uint64_t table_uploads;   /* whole-table uploads of the device copy */
  uint64_t table_merges;    /* incremental device updates (merge kernel) */
} cg_stats;

/* ------------------------------------------------------------- lifetime */

/* Fill *cfg with the defaults. */
cg_status cg_config_default(cg_config *cfg);

/* Create a context on the current CUDA device.  cfg may be NULL (defaults).
 * Owns: the allocation table (host mirror + device copy), the device V
 * shadow pool, small device scratch and pinned staging buffers. */
cg_status cg_create(cg_ctx **out, const cg_config *cfg);

/* Synchronises the context's work and frees everything it owns. */
cg_status cg_destroy(cg_ctx *ctx);

/* Bind the host shadow image (Memcheck's A and V bits of host memory,
 * Sec. 1.1).  a_bits_dev: n_bytes/8 bytes; v_dev: n_bytes bytes; each in
 * device memory, managed memory, or pinned host memory mapped into the
 * device (then read in place over the host link, with register loads).
 * Both 16-byte aligned; n_bytes a multiple of 128 (so both arrays are whole
 * 16-byte vectors).  The caller keeps ownership and must keep them alive
 * while bound; DtoH checks write v_dev (the carry).  Rebinding replaces the
 * previous image.  CG_E_ALIGN on a broken rule, CG_E_ARG for memory the
 * device cannot read. */
cg_status cg_bind_host_shadow(cg_ctx *ctx, const uint8_t *a_bits_dev,
                              uint8_t *v_dev, uint64_t n_bytes);

/* Copy host-side shadow bytes [off, off+n) of an image held in host memory
 * (pinned for speed) into the bound device image: V bytes [off, off+n) and
 * A bytes [off/8, (off+n)/8).  off and n multiples of 8.  Asynchronous on
 * `stream`; the host buffers must stay valid until the stream reaches it. */
cg_status cg_upload_host_shadow(cg_ctx *ctx, const uint8_t *a_bits_host,
                                const uint8_t *v_host, uint64_t off,
                                uint64_t n, void *stream);

/* --------------------------------------------------- allocation table */

/* Record a device allocation [dptr, dptr+size) (the cuMemAlloc wrapper's
 * bookkeeping, Fig. 2).  Its V shadow starts all undefined.  Frees bases
 * it covers from the freed set.  CG_E_ZERO_SIZE, CG_E_WRAP, CG_E_OVERLAP
 * (table unchanged), CG_E_NOMEM (shadow pool exhausted or over budget). */
cg_status cg_register_alloc(cg_ctx *ctx, uint64_t dptr, uint64_t size);

/* Register many; st_out[i] (host, may be NULL) gets each status.  Returns
 * CG_OK if all succeeded, else the first failure's status. */
cg_status cg_register_allocs(cg_ctx *ctx, const uint64_t *dptr,
                             const uint64_t *size, uint64_t count,
                             cg_status *st_out);

/* The cuMemFree wrapper's check: *verdict gets CG_FREE_OK (allocation
 * removed, its shadow released), CG_FREE_INTERIOR, CG_FREE_DOUBLE or
 * CG_FREE_UNKNOWN (table unchanged for the last three). */
cg_status cg_free(cg_ctx *ctx, uint64_t dptr, uint32_t *verdict);

/* Memcheck-style client requests on device memory: mark [dptr, dptr+n) as
 * defined (V = 0) or undefined (V = 0xFF), e.g. a kernel's output.  The
 * range must lie in one live allocation (CG_E_RANGE).  Asynchronous. */
cg_status cg_mark_defined(cg_ctx *ctx, uint64_t dptr, uint64_t n, void *stream);
cg_status cg_mark_undefined(cg_ctx *ctx, uint64_t dptr, uint64_t n, void *stream);

/* Copy the device V shadow of [dptr, dptr+n) (one live allocation) into
 * host memory `out`.  Synchronous.  CG_E_RANGE otherwise. */
cg_status cg_read_device_shadow(cg_ctx *ctx, uint64_t dptr, uint64_t n,
                                uint8_t *out);

/* ---------------------------------------------------------------- checks */

/* Check one copy and carry its V shadow (Sec. 2 itemize, Listing 5,
 * Sec. 5).  req, rep: host.  Synchronous: returns once *rep is filled.
 * API errors: CG_E_KIND, CG_E_HOST_RANGE, CG_E_NO_HOST (HtoD/DtoH with no
 * image bound); nothing is checked or carried then. */
cg_status cg_check_copy(cg_ctx *ctx, const cg_copy *req, cg_report *rep,
                        void *stream);

/* The same check, enqueued on `stream` without waiting: the report is
 * written to rep_dev (device memory, or mapped pinned host memory) when
 * the stream reaches it.  Validation and the allocation lookup use the
 * table as it is at call time.  Checks of one context must all be
 * enqueued on one stream (they share a small device scratch area and the
 * staging buffer for overlapping device->device copies). */
cg_status cg_check_copy_async(cg_ctx *ctx, const cg_copy *req, cg_report *rep_dev,
                              void *stream);

/* Check copies reqs[0..nreq) with the result of checking them one after
 * another in order (the same reports, records and final shadow state).
 * Independent copies run together: one persistent kernel per dependency
 * level over byte segments of all copies of the level.  reqs, reps, recs,
 * n_rec: host.  reps may be NULL; recs may be NULL when rec_cap is 0.
 * *n_rec gets the total record count, which may exceed rec_cap (then only
 * the first rec_cap records are written).  Synchronous.  A batch holding an
 * invalid request is refused as a whole (*n_rec untouched, nothing runs);
 * *bad_index (may be NULL) gets its index. */
cg_status cg_check_batch(cg_ctx *ctx, const cg_copy *reqs, uint64_t nreq,
                         cg_report *reps, cg_err_record *recs,
                         uint64_t rec_cap, uint64_t *n_rec,
                         uint64_t *bad_index, void *stream);

/* The same batch check, returned from as soon as it is enqueued: *ticket
 * identifies it for cg_batch_wait.  Two batches may be in flight per
 * context (CG_E_FULL for a third).  A batch's device lookup runs on a
 * stream of the context's own and its level plan on the host while the
 * batch before it still runs on `stream`; its kernels follow that batch's
 * on `stream`, so batches take effect in submission order, with exactly
 * the results of cg_check_batch called in that order.  The request array
 * is copied before return.  rec_cap bounds the records kept on the device
 * for this batch.  Errors as cg_check_batch (nothing is enqueued then). */
cg_status cg_check_batch_async(cg_ctx *ctx, const cg_copy *reqs, uint64_t nreq,
                               uint64_t rec_cap, uint64_t *ticket, uint64_t *bad_index,
                               void *stream);

/* Wait for the batch `ticket` and write its reports (reps, may be NULL), up
 * to rec_cap records (recs) and the total record count (*n_rec, may be
 * NULL); host buffers.  CG_E_ARG for an unknown or already collected
 * ticket; CG_E_TIMEOUT as cg_check_batch. */
cg_status cg_batch_wait(cg_ctx *ctx, uint64_t ticket, cg_report *reps, cg_err_record *recs,
                        uint64_t rec_cap, uint64_t *n_rec);

/* ------------------------------------------- pitched copies and arrays */

/* One side of a pitched 2-D / 3-D copy (cuMemcpy2D / cuMemcpy3D).  ptr is a
 * device address, a host offset into the bound image (the host side of
 * CG_HTOD / CG_DTOH), or, with is_array = 1, the handle of a device array
 * registered with cg_register_array.  pitch = bytes between rows, rows =
 * rows per slice, (x, y, z) = the origin, x in bytes.  For an array side,
 * pitch and rows are ignored: the array's own width and height apply.
 * reserved must be 0.  56 bytes. */
typedef struct cg_side3d {
  uint64_t ptr;
  uint64_t pitch;
  uint64_t rows;
  uint64_t x, y, z;
  uint32_t is_array;
  uint32_t reserved;
} cg_side3d;

/* A pitched copy of depth slices of height rows of width bytes.  Byte
 * (i, y, z) of the copy (i < width, y < height, z < depth) lives at
 *   ptr + (z0+z)*pitch*rows + (y0+y)*pitch + x0+i   (linear memory, host)
 *   dense position ((z0+z)*H + y0+y)*W + x0+i        (a W x H x D array)
 * on each side, (x0, y0, z0) being that side's origin.  Rules (Sec. 2, its
 * footnote on strided host access, Fig. 2):
 *   - only the copied bytes are classified, never a pitch gap; report
 *     offsets are linear in the copy, (z*height + y)*width + i, and
 *     expected = width*height*depth;
 *   - a linear device side must hold its whole extent, first to one past
 *     the last copied byte, in one live allocation (found and alloc_* as
 *     for a plain copy, measured from the first copied byte);
 *   - an array side must name a live array and fit per dimension
 *     (x0+width <= W, y0+height <= H, z0+depth <= D), else OVERRUN; found =
 *     W*H*D minus the origin's dense position (0 if the origin lies
 *     outside), alloc_base = the handle, alloc_size = W*H*D;
 *   - device->device: the overlap warning is raised when the two spans
 *     intersect (arrays: the same array); the carry reads the whole source
 *     first.
 * reserved must be 0.  144 bytes. */
typedef struct cg_copy3d {
  uint32_t kind;
  uint32_t reserved;
  cg_side3d dst;
  cg_side3d src;
  uint64_t width;
  uint64_t height;
  uint64_t depth;
} cg_copy3d;

/* Register a device array (Fig. 2's second list: the cuArrayCreate /
 * cuArray3DCreate wrapper): handle = the array's handle, width in bytes,
 * height and depth >= 1.  Its shadow is dense, row-major, all undefined.
 * Handles are a namespace of their own (no clash with device addresses).
 * CG_E_ZERO_SIZE, CG_E_WRAP (W*H*D beyond 64 bits), CG_E_OVERLAP (handle
 * already live), CG_E_NOMEM. */
cg_status cg_register_array(cg_ctx *ctx, uint64_t handle, uint64_t width, uint64_t height,
                            uint64_t depth);

/* The cuArrayDestroy wrapper's check: *verdict = CG_FREE_OK (removed,
 * shadow released), CG_FREE_DOUBLE (destroyed before and not re-created)
 * or CG_FREE_UNKNOWN. */
cg_status cg_free_array(cg_ctx *ctx, uint64_t handle, uint32_t *verdict);

/* Copy bytes [off, off+n) of an array's dense shadow to host memory `out`.
 * Synchronous.  CG_E_RANGE if the handle is not live or the span is
 * outside the array. */
cg_status cg_read_array_shadow(cg_ctx *ctx, uint64_t handle, uint64_t off, uint64_t n,
                               uint8_t *out);

/* Check one pitched copy and carry its V shadow.  req, rep: host.
 * Synchronous.  API errors, checked in this order (nothing runs then):
 * CG_E_KIND; CG_E_ARG (reserved fields, an array as the host side);
 * CG_E_WRAP (width*height*depth beyond 64 bits); then, for a non-empty
 * copy, CG_E_ARG (pitch < width with height or depth > 1, rows < height
 * with depth > 1), CG_E_NO_HOST, CG_E_WRAP (a position or extent beyond
 * 64 bits), CG_E_HOST_RANGE (the host extent outside the image).  An
 * empty copy is a no-op (expected 0, no range check). */
cg_status cg_check_copy3d(cg_ctx *ctx, const cg_copy3d *req, cg_report *rep, void *stream);

/* Asynchronous form (as cg_check_copy_async): the report is written to
 * rep_dev when `stream` reaches it. */
cg_status cg_check_copy3d_async(cg_ctx *ctx, const cg_copy3d *req, cg_report *rep_dev,
                                void *stream);

/* --------------------------------------- memset and kernel arguments */

/* The memset wrappers' check (cuMemsetD8/D16/D32 and cuMemsetD2D8/16/32:
 * every driver call that writes device memory is wrapped, Sec. 2): height
 * rows of width BYTES (elements x element size) at dptr + y*pitch.  The
 * extent (height-1)*pitch + width must lie in one live allocation
 * (UNALLOC_DST / OVERRUN_DST, found_dst and alloc_*_dst as for a copy);
 * with carry on, the written bytes then become defined (V = 0).  expected =
 * n_good = width*height (nothing is read).  width*height == 0 is a no-op.
 * API errors: CG_E_ARG (pitch < width with height > 1), CG_E_WRAP.  *rep
 * (host) is final at return; the shadow update is enqueued on `stream`. */
cg_status cg_check_memset(cg_ctx *ctx, uint64_t dptr, uint64_t pitch, uint64_t width,
                          uint64_t height, cg_report *rep, void *stream);

/* The same, with the report written to rep_dev (device or mapped pinned
 * memory) when `stream` reaches it. */
cg_status cg_check_memset_async(cg_ctx *ctx, uint64_t dptr, uint64_t pitch, uint64_t width,
                                uint64_t height, cg_report *rep_dev, void *stream);

/* One pointer argument of a kernel launch (the cuLaunchKernel wrapper of
 * the paper's outlook, Sec. 5.1): the device pointer, the bytes the kernel
 * may touch from it, and how (CG_ARG_READ, CG_ARG_WRITE or both).
 * reserved must be 0.  24 bytes. */
#define CG_ARG_READ 1u  /* reads [ptr, ptr+bytes): undefined bytes are reported */
#define CG_ARG_WRITE 2u /* writes all of [ptr, ptr+bytes): it becomes defined */
typedef struct cg_karg {
  uint64_t ptr;
  uint64_t bytes;
  uint32_t access;
  uint32_t reserved;
} cg_karg;

/* Check the pointer arguments args[0..nargs) of one launch, one report
 * each (reps: host, may be NULL).  A read argument is checked as a copy
 * source (UNALLOC_SRC / OVERRUN_SRC, found_src, alloc_*_src) and, in range,
 * its undefined device bytes are counted (n_undef, first_undef_off, the
 * DEV_UNDEF_SRC warning, an error in strict mode); a write argument as a
 * destination (UNALLOC_DST / OVERRUN_DST).  bytes == 0: only that the
 * pointer lies in a live allocation.  Every read sees the state before the
 * launch; then, with carry on, every write argument in range becomes
 * defined over its whole range.  expected = bytes, n_good = bytes -
 * n_undef.  Synchronous.  CG_E_ARG (an access outside READ|WRITE, or 0;
 * reserved != 0) refuses the whole call, *bad_index (may be NULL) = the
 * argument. */
cg_status cg_check_kernel_args(cg_ctx *ctx, const cg_karg *args, uint64_t nargs,
                               cg_report *reps, uint64_t *bad_index, void *stream);

/* ------------------------------------------------ choosing the batch split */

/* How cg_check_batch cuts copies into segments matters (too small: per-
 * segment overhead; too large: idle warps at the end of each level), and
 * the best size depends on the batch.  With batch_segment_kib = 0 the
 * context picks it per batch, in this order: the size measured best for a
 * batch with close features (by cg_tune_batch, or by the online tuner);
 * with batch_autotune on, the next candidate the online tuner wants to
 * try for this shape; the argmin of a learned cost model over the
 * candidates 4, 8, ..., 1024 KiB; else 64 KiB. */

#define CG_NFEAT 13

/* Features of a batch (host only): [0] log2(1+count), [1] mean and [2]
 * standard deviation of log2(1+n), [3..8] fraction of all bytes in copies
 * of at most 4 KiB, 64 KiB, 1 MiB, 4 MiB, 16 MiB, and above, [9..11]
 * fraction of HtoD, DtoH, DtoD copies, [12] log2(1+total bytes). */
cg_status cg_batch_features(const cg_copy *reqs, uint64_t nreq, float *feat);

/* Autotuner: time the batch's level kernels for each candidate segment
 * size (seg_kib[0..ncand), or the default candidates when seg_kib is NULL,
 * then ms gets ncand or 9 entries) `repeats` times each and keep the
 * fastest.  With flags & CG_TUNE_REMEMBER the best size is remembered for
 * batches with these features.  Trial runs are dry (the carry is masked
 * off: no shadow changes), so tuning may run on the live context.
 * Synchronous. */
#define CG_TUNE_REMEMBER 1u
cg_status cg_tune_batch(cg_ctx *ctx, const cg_copy *reqs, uint64_t nreq, const uint32_t *seg_kib,
                        uint32_t ncand, uint32_t repeats, uint32_t flags, float *ms,
                        uint32_t *best_kib, void *stream);

/* Install a learned cost model (NULL or hidden = 0 removes it): a
 * one-hidden-layer ReLU network predicting log2(batch milliseconds) from
 * x = (features, log2(segment KiB)), D = CG_NFEAT + 1 inputs.  weights (host,
 * copied): mu[D], sigma[D] (inputs are standardised (x - mu) / sigma),
 * W1[D][hidden] row-major, b1[hidden], w2[hidden], b2. */
cg_status cg_set_cost_model(cg_ctx *ctx, const float *weights, uint32_t hidden);

/* Fit the cost model on the GPU (this library's own forward and backward
 * kernels, full-batch Adam, mean squared error): x[n][D] raw inputs and
 * t[n] targets (log2 ms), host.  hidden: a multiple of 32, at most 1024.
 * weights (host) receives the cg_set_cost_model layout, including the
 * standardisation fitted to x; losses (host, may be NULL) gets the loss
 * before each of the `epochs` steps.  Synchronous. */
cg_status cg_mlp_fit(const float *x, const float *t, uint32_t n, uint32_t hidden,
                     uint32_t epochs, float lr, uint64_t seed, float *weights, float *losses,
                     void *stream);

/* One forward and backward pass on the GPU with the given weights (the
 * cg_set_cost_model layout): grads (same layout; zero for mu and sigma)
 * and the mean squared error *loss.  For checking the kernels. */
cg_status cg_mlp_grad(const float *x, const float *t, uint32_t n, uint32_t hidden,
                      const float *weights, float *grads, float *loss, void *stream);

/* The segment size cg_check_batch would use for this batch; *source (may be
 * NULL): 0 default, 1 tuned entry, 2 learned model, 3 fixed by the config,
 * 4 an online-tuning trial. */
cg_status cg_choose_segment(const cg_ctx *ctx, const cg_copy *reqs, uint64_t nreq,
                            uint32_t *seg_kib, uint32_t *source);

/* The tuned split entries the context holds (batch features -> segment
 * KiB, from cg_tune_batch with CG_TUNE_REMEMBER or finished online trials),
 * for saving: up to cap entries into feat (cap * CG_NFEAT floats) and kib
 * (host); *count gets how many there are. */
cg_status cg_get_tuned(const cg_ctx *ctx, float *feat, uint32_t *kib, uint32_t cap,
                       uint32_t *count);

/* Add tuned entries (e.g. saved from an earlier run): count entries of
 * CG_NFEAT features and a segment size in KiB (> 0) each. */
cg_status cg_add_tuned(cg_ctx *ctx, const float *feat, const uint32_t *kib, uint32_t count);

/* --------------------------------------------------------------- serving */

/* A serving loop in the context: client threads submit requests into
 * per-client rings as they arrive; one scheduler thread admits them in one
 * global order (result.seq), applies allocation events to the table at
 * their place in that order, and packs the checks that arrive while others
 * are on the GPU into rounds ("continuous batching").  A round is planned
 * like cg_check_batch (dependency levels) and runs on one of `streams`
 * streams; rounds overlap on the device unless one touches shadow another
 * in-flight round touches, in which case it waits for that round.
 * Admission stops while the bytes of admitted, unfinished checks would
 * exceed budget_bytes.  Every result equals the one the same request gets
 * when all requests are applied one by one in seq order (cg_check_copy,
 * cg_register_alloc, cg_free, cg_mark_*), except for one finding only
 * serving can make: the paper's concurrent accesses of several threads
 * (Sec. 2 itemize).  A check r gets CG_F_CONCURRENT (a warning; race_seq =
 * the smallest such seq) when a copy q of another client, admitted before
 * r, had not yet returned its result when r was submitted (q.done_ns >
 * r.submit_ns), and one of them writes data the other reads or writes:
 * the data ranges [dst, dst+n) written and [src, src+n) read, host offsets
 * and device addresses apart, of copies whose device ranges are valid.
 * Sec. 2's wrappers check each call as it happens; serving keeps that
 * order while batching the work. */

#define CG_OP_CHECK 1u
#define CG_OP_ALLOC 2u          /* dst = base, n = size */
#define CG_OP_FREE 3u           /* dst = base */
#define CG_OP_MARK_DEFINED 4u   /* dst, n */
#define CG_OP_MARK_UNDEFINED 5u /* dst, n */

#define CG_PENDING 1 /* cg_poll: the result is not ready yet (not an error) */

typedef struct cg_request {
  uint32_t op;   /* CG_OP_* */
  uint32_t kind; /* CG_OP_CHECK: the copy kind */
  uint64_t dst;
  uint64_t src;
  uint64_t n;
} cg_request; /* 32 bytes */

typedef struct cg_result {
  uint64_t seq;       /* place in the global order the request took effect in */
  int32_t status;     /* CG_OK or the request's own API error */
  uint32_t verdict;   /* CG_OP_FREE: CG_FREE_* */
  uint64_t submit_ns; /* steady clock at cg_submit */
  uint64_t done_ns;   /* steady clock when the result became visible */
  cg_report report;   /* CG_OP_CHECK */
} cg_result; /* 152 bytes */

typedef struct cg_serve_config {
  uint32_t clients;       /* client rings, 1..64 (0 = 8) */
  uint32_t ring_capacity; /* requests per client, a power of two (0 = 4096) */
  uint32_t max_round;     /* checks per round at most (0 = 8192) */
  uint32_t streams;       /* rounds on the GPU at once, 1..8 (0 = 4) */
  uint64_t budget_bytes;  /* bytes of admitted, unfinished checks (0 = 8 GiB);
                             a single larger check is still admitted alone */
  uint32_t reserved[10];
} cg_serve_config;

typedef struct cg_serve_stats {
  uint64_t requests;       /* admitted */
  uint64_t checks;
  uint64_t rounds;
  uint64_t round_checks_max;
  uint64_t conflict_waits; /* rounds that had to wait for an in-flight round */
  uint64_t budget_stalls;  /* admissions stopped by the budget */
  uint64_t bytes_checked;
  uint64_t inflight_bytes_max;
} cg_serve_stats;

/* Start serving.  While serving, the context accepts only cg_submit,
 * cg_poll, cg_wait, cg_serve_replay, cg_get_stats and cg_serve_stop
 * (CG_E_STATE otherwise).  Allocates the rings and per-stream round
 * buffers and starts the scheduler thread. */
cg_status cg_serve_start(cg_ctx *ctx, const cg_serve_config *cfg);

/* Submit one request from client `client` (0..clients-1).  Each client
 * index must be driven by one thread at a time (cg_submit and cg_poll /
 * cg_wait of its tickets).  *ticket identifies the result.  CG_E_FULL when
 * the client has ring_capacity requests submitted and not yet collected. */
cg_status cg_submit(cg_ctx *ctx, uint32_t client, const cg_request *req, uint64_t *ticket);

/* Collect a result: CG_OK (copied to *out, ticket released), CG_PENDING,
 * or CG_E_ARG for an unknown or already collected ticket. */
cg_status cg_poll(cg_ctx *ctx, uint64_t ticket, cg_result *out);

/* cg_poll until done or timeout_ms pass (CG_E_TIMEOUT). */
cg_status cg_wait(cg_ctx *ctx, uint64_t ticket, uint32_t timeout_ms, cg_result *out);

/* Replay a timed trace: request i is submitted by client client[i] at
 * arrival_ns[i] after the call starts (one host thread per client; each
 * client's requests in index order), and its result lands in results[i].
 * Returns once every result is in.  Host arrays. */
cg_status cg_serve_replay(cg_ctx *ctx, const cg_request *reqs, const uint32_t *client,
                          const uint64_t *arrival_ns, uint64_t n, cg_result *results);

/* Finish the admitted work, stop the scheduler, free the serving buffers.
 * out (may be NULL) gets the serving counters. */
cg_status cg_serve_stop(cg_ctx *ctx, cg_serve_stats *out);

/* --------------------------------------------- allocation-free variant */

/* The paper has no counterpart to this entry point; it exists for callers
 * that must not allocate device memory.  A checker that runs inside a
 * program's own allocation and copy calls (an interposer around the
 * driver's memory functions, as the paper's wrappers are) cannot call
 * cudaMalloc without re-entering the allocator it wraps, and a process
 * whose device memory is owned by another allocator may have none to give.
 * cg_create allocates; this call does not: no cudaMalloc, cudaFree or other
 * allocating routine, and no context.
 *
 * It runs the single-copy scan of cg_check_copy (per-byte classes, counts,
 * first offsets, and the V carry when carry != 0) over buffers the caller
 * passes; there is no allocation table, so the report's range fields
 * (found_*, alloc_*, UNALLOC/OVERRUN flags) stay zero.
 *   kind            CG_HTOD, CG_DTOH or CG_DTOD
 *   a_bits_dev,     host shadow image as in cg_bind_host_shadow (device,
 *   host_v_dev,     16-byte aligned, host_n a multiple of 128); unused and
 *   host_n          may be NULL/0 for CG_DTOD
 *   host_off        offset of the copy in the host image (HtoD source,
 *                   DtoH destination)
 *   dev_src_shadow  device V shadow of the source bytes (DtoH/DtoD); NULL =
 *                   source definedness unknown (not counted, no carry)
 *   dev_dst_shadow  device V shadow receiving the carry (HtoD/DtoD); NULL =
 *                   no carry
 *   rep_dev         device memory (or mapped pinned host memory) receiving
 *                   the report when the stream reaches it
 * Device shadows must be device (or managed) memory, else CG_E_ARG; they
 * are read in whole 16-byte-aligned blocks around [ptr, ptr+n) (those
 * blocks must be readable); only [ptr, ptr+n) is written.
 *
 * Its scratch (the kernel's accumulators and an 8 MiB staging area for an
 * overlapping device->device carry) is a fixed array inside the library
 * that every GPU loading libcg holds until the process exits.  An
 * overlapping device->device carry above 8 MiB is refused (CG_E_TOO_BIG).
 * Every call shares that array and the accumulators are reset at the start
 * of each call, so calls whose work overlaps on the GPU (e.g. on two
 * streams, or from two threads) race and their reports are wrong: order
 * them on one stream.  The first call on each device looks up the array's
 * device address (cudaGetSymbolAddress, no allocation); make that first
 * call before any stream capture.  Asynchronous; errors as cg_check_copy,
 * plus CG_E_TOO_BIG, with text in cg_last_error(). */
cg_status cg_scan_noalloc(uint32_t kind, const uint8_t *a_bits_dev, uint8_t *host_v_dev,
                          uint64_t host_n, uint64_t host_off, const uint8_t *dev_src_shadow,
                          uint8_t *dev_dst_shadow, uint64_t n, uint32_t carry,
                          cg_report *rep_dev, void *stream);

/* ------------------------------------------------------ checkpoint / resume */

/* Save the context's checking state to the file `path`: every live
 * allocation with its device V shadow, the freed bases (so double frees are
 * still recognised), the device arrays with their shadows and the destroyed
 * array handles.  The host shadow image is the caller's and is not saved.
 * Synchronous; CG_E_ARG with text in cg_last_error() when the file cannot
 * be written. */
cg_status cg_snapshot(cg_ctx *ctx, const char *path);

/* Load a snapshot into a context that has no allocations, freed bases or
 * arrays yet (CG_E_STATE otherwise); its configuration is the context's own.
 * After it, checks give the results they would have given in the saved
 * context.  CG_E_ARG for a file that is not a complete snapshot (the
 * context may then hold part of it). */
cg_status cg_restore(cg_ctx *ctx, const char *path);

/* ------------------------------------------------------- fault injection */

/* Host-side hooks that make one failure happen on purpose, so that the
 * error paths can be tested without faulting a GPU.  One-shot: the fault
 * applies to the next operation that can take it, then is cleared.
 *   CG_FAULT_STALL_COPY: the next single check that runs on the TMA engine
 *     never issues one of its bulk copies, so the wait for that tile runs
 *     out (about one second, %globaltimer): the report carries
 *     CG_F_INCOMPLETE and cg_check_copy returns CG_E_TIMEOUT.  No copy is
 *     left in flight; the context stays usable.
 *   CG_FAULT_SHADOW_ALLOC: the next shadow allocation fails:
 *     cg_register_alloc / cg_register_array return CG_E_NOMEM and the table
 *     is unchanged. */
#define CG_FAULT_NONE 0u
#define CG_FAULT_STALL_COPY 1u
#define CG_FAULT_SHADOW_ALLOC 2u
cg_status cg_inject_fault(cg_ctx *ctx, uint32_t fault);

/* ----------------------------------------------------------- diagnostics */

/* The dependency levels cg_check_batch runs reqs[0..nreq) in (host only,
 * no GPU work): level[i] = 1 + the highest level of an earlier request that
 * reads what request i writes, writes what it reads, or writes what it
 * writes; 0 when there is none, and all 0 when carry is 0.  modes (host,
 * may be NULL) gives per request bit 0 = it carries (writes its
 * destination's V), bit 1 = its device source is valid (its V is read);
 * cg_check_batch passes the values its device lookup found.  With NULL,
 * every request is taken to read its source and write its destination.
 * reqs, level: host.  *n_levels (may be NULL) gets 1 + the highest level. */
cg_status cg_plan_levels(const cg_copy *reqs, uint64_t nreq, uint32_t carry,
                         const uint8_t *modes, int32_t *level, uint32_t *n_levels);

/* The planning units cg_check_batch runs a batch as on the TMA engine
 * (host only, no GPU work): every copy is one unit, except host->device
 * copies that carry nothing (their modes bit 0 clear) and span more than
 * 1.5 x piece_rows rows of their anchor grid (512 host bytes a row, the
 * grid starting at the 16-byte boundary at or below src): those are cut
 * into units of piece_rows rows (the last one shorter).  Each unit gets a
 * level: 1 + the highest level of an earlier unit it conflicts with (as in
 * cg_plan_levels; in the host space exact unless a 64 KiB block of the host
 * image holds more than 8 ranges that cover it in part: then units
 * touching that block are taken to conflict).  host_n: the host image's size
 * (host ranges must lie inside it).  Output per unit, in request order
 * (host arrays of cap entries): req, rows [row_lo, row_hi) (0, 0: the
 * whole copy), level; *n_units gets the count (units beyond cap are not
 * written; CG_E_TOO_BIG if there are more than cap). */
cg_status cg_plan_units(const cg_copy *reqs, uint64_t nreq, uint32_t carry,
                        const uint8_t *modes, uint64_t host_n, uint64_t piece_rows,
                        uint32_t *req, uint32_t *row_lo, uint32_t *row_hi, int32_t *level,
                        uint64_t cap, uint64_t *n_units);

cg_status cg_get_stats(const cg_ctx *ctx, cg_stats *out);

/* The allocation table as the device copy holds it, brought up to date
 * first (an incremental merge on the device, or a whole upload): up to cap
 * entries into base, size and shadow (host arrays, shadow may be NULL) in
 * base order; *count gets the number of live entries.  Synchronises
 * `stream`.  Not allowed while serving or with batches in flight. */
cg_status cg_device_table(cg_ctx *ctx, uint64_t *base, uint64_t *size, uint64_t *shadow,
                          uint64_t cap, uint64_t *count, void *stream);

/* Text for a report, e.g. for a device->host overrun:
 *   "device->host copy of 8000000 bytes overruns its source allocation:
 *    only 4000000 bytes from the pointer to its end"
 * Writes at most cap bytes (NUL-terminated); returns CG_OK. */
cg_status cg_format_report(const cg_report *rep, uint32_t kind, char *buf,
                           size_t cap);

/* The last CUDA or internal error message of this thread ("" if none). */
const char *cg_last_error(void);

/* Library version, e.g. "0.1.0". */
const char *cg_version(void);

#ifdef __cplusplus
}
#endif
#endif /* CG_H */

/*
 * cg_oracle.h -- plain, byte-by-byte CPU checker for Cudagrind-style transfer
 * checks (Baumann & Gracia, "Cudagrind: A Valgrind Extension for CUDA").
 *
 * TEST INFRASTRUCTURE ONLY.  This checker exists to prove the GPU library
 * right.  Only the test suite, the smoke check and the benchmark's CPU
 * baseline may load it; the product path never does.  It shares no code,
 * header, constant table or helper with the GPU library: every definition
 * below is written here again on purpose.
 *
 * What it models (the paper's Sec. 2 itemize and Fig. 2 caption):
 *   - a list of live device allocations (base, size), with a device
 *     definedness shadow (one V byte per device byte, 0xFF = undefined);
 *   - a host shadow image: a packed addressability bitmap (A, 1 bit per byte,
 *     LSB first, 1 = addressable) and a definedness mask (V, 1 byte per byte,
 *     bit b set = data bit b undefined);
 *   - copy checks host->device, device->host and device->device (Sec. 5),
 *     frees of unknown / already freed / interior pointers.
 */
#ifndef CG_ORACLE_H
#define CG_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* copy kinds */
#define OR_HTOD 1u
#define OR_DTOH 2u
#define OR_DTOD 3u

/* per-byte classes */
#define OR_BYTE_GOOD   0u
#define OR_BYTE_UNADDR 1u
#define OR_BYTE_UNDEF  2u

/* report flag bits; record classes are the bit indices */
#define OR_F_UNALLOC_DST  (1u << 0)
#define OR_F_UNALLOC_SRC  (1u << 1)
#define OR_F_OVERRUN_DST  (1u << 2)
#define OR_F_OVERRUN_SRC  (1u << 3)
#define OR_F_HOST_UNADDR  (1u << 4)
#define OR_F_HOST_UNDEF   (1u << 5)
#define OR_F_DEV_UNDEF_SRC (1u << 6)
#define OR_F_DTOD_OVERLAP (1u << 7)
#define OR_F_CONCURRENT (1u << 8)
#define OR_NFLAGS 9

/* free verdicts */
#define OR_FREE_OK       0u
#define OR_FREE_UNKNOWN  1u
#define OR_FREE_DOUBLE   2u
#define OR_FREE_INTERIOR 3u

/* status codes */
#define OR_OK            0
#define OR_E_ARG        -1
#define OR_E_KIND       -2
#define OR_E_HOST_RANGE -3
#define OR_E_ZERO_SIZE  -4
#define OR_E_WRAP       -5
#define OR_E_OVERLAP    -6
#define OR_E_NOMEM      -7
#define OR_E_RANGE      -8

typedef struct or_report {
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
  int64_t race_seq;
} or_report;

typedef struct or_record {
  uint64_t req;
  uint32_t cls;
  uint32_t severity; /* 0 error, 1 warning */
  int64_t off;
  uint64_t count;
  uint64_t expected;
  uint64_t found;
} or_record;

typedef struct or_state or_state;

/* The host images are copied in; carry != 0 enables V-shadow propagation,
 * strict != 0 makes undefined device-source bytes an error, not a warning. */
or_state *or_create(uint64_t host_n, const uint8_t *a_bits, const uint8_t *v,
                    int carry, int strict);
void or_destroy(or_state *s);

int or_register_alloc(or_state *s, uint64_t base, uint64_t size);
/* or_register_alloc applied to each (bases[i], sizes[i]) in turn, its
 * status in status[i]; returns the number of refused registrations. */
uint64_t or_register_allocs(or_state *s, const uint64_t *bases, const uint64_t *sizes,
                            uint64_t n, int32_t *status);
int or_free(or_state *s, uint64_t base, uint32_t *verdict);
int or_mark(or_state *s, uint64_t dptr, uint64_t n, uint8_t value);

int or_check_copy(or_state *s, uint32_t kind, uint64_t dst, uint64_t src,
                  uint64_t n, or_report *rep);
/* requests in order; the whole batch is rejected if any request is invalid */
int or_check_batch(or_state *s, const uint32_t *kind, const uint64_t *dst,
                   const uint64_t *src, const uint64_t *n, uint64_t nreq,
                   or_report *reps, uint64_t *bad_index);

/* Pitched 2-D / 3-D copies and device arrays (Sec. 2: the context keeps a
 * list of linear allocations and one of device arrays, Fig. 2; the footnote
 * to the error list: strided host access is not an error).
 *
 * A copy moves depth slices of height rows of width bytes.  On each side,
 * byte (i, y, z) of the copy (i < width, y < height, z < depth) lives at
 *   linear memory / host image:  ptr + (z0+z)*pitch*rows + (y0+y)*pitch + x0+i
 *   device array (ptr = handle): shadow[((z0+z)*H + y0+y)*W + x0+i]
 * where (x0, y0, z0) = (x, y, z) of the side (x in bytes), pitch = bytes per
 * row, rows = rows per slice, and W x H x D the array's dimensions.
 * pitch >= width when height > 1 or depth > 1, rows >= height when depth > 1
 * (OR_E_ARG otherwise); both still place the origin when they are not
 * needed for the rows themselves.
 * Linear device sides: the extent from the first to one past the last
 * copied byte lies in one live allocation.  Array sides: the handle is a
 * live array and x0+width <= W, y0+height <= H, z0+depth <= D; found = the
 * array bytes from the origin's dense position to the end (0 if the origin
 * is outside).  Only copied bytes are classified (a pitch gap never is), at
 * offsets (z*height + y)*width + i; expected = width*height*depth.  The host
 * side is never an array (OR_E_ARG). */
typedef struct or_side3d {
  uint64_t ptr; /* device address, host image offset, or array handle */
  uint64_t pitch;
  uint64_t rows;
  uint64_t x, y, z;
  uint32_t is_array;
  uint32_t reserved;
} or_side3d;

typedef struct or_copy3d {
  uint32_t kind;
  uint32_t reserved;
  or_side3d dst, src;
  uint64_t width, height, depth;
} or_copy3d;

int or_check_copy3d(or_state *s, const or_copy3d *q, or_report *rep);
int or_register_array(or_state *s, uint64_t handle, uint64_t w, uint64_t h, uint64_t d);
/* verdict: OR_FREE_OK, OR_FREE_DOUBLE (destroyed before) or OR_FREE_UNKNOWN */
int or_free_array(or_state *s, uint64_t handle, uint32_t *verdict);
/* bytes [off, off+n) of an array's dense shadow */
int or_read_array_v(const or_state *s, uint64_t handle, uint64_t off, uint64_t n, uint8_t *out);

/* The memset wrappers (cuMemsetD8/16/32 and their 2-D forms; Sec. 2 wraps
 * every driver call that touches device memory): height rows of width bytes
 * at dptr + y*pitch (pitch >= width when height > 1, else OR_E_ARG).  The
 * extent (height-1)*pitch + width must lie in one live allocation
 * (UNALLOC_DST / OVERRUN_DST, found_dst as for a copy); then, with carry on,
 * every written byte becomes defined.  expected = n_good = width*height
 * (nothing is read).  width*height == 0 is a no-op. */
int or_memset(or_state *s, uint64_t dptr, uint64_t pitch, uint64_t width, uint64_t height,
              or_report *rep);

/* Kernel launch arguments (Sec. 5.1, Outlook: a cuLaunchKernel wrapper that
 * checks the pointers a kernel is given).  Argument i: device pointer
 * ptr[i], the bytes[i] the kernel may touch from there, access[i] = a
 * nonzero subset of OR_ARG_READ | OR_ARG_WRITE (else OR_E_ARG, nothing
 * done).  A read argument is checked as a copy source (UNALLOC_SRC /
 * OVERRUN_SRC, found_src, alloc_*_src) and, when in range, its undefined
 * device bytes are counted (n_undef, first_undef_off, DEV_UNDEF_SRC); a
 * write argument as a destination (UNALLOC_DST / OVERRUN_DST).  bytes[i] ==
 * 0 checks only that the pointer lies in a live allocation.  Every read
 * sees the state before the launch; then (carry on) each write argument
 * with a valid range becomes defined over its whole range.
 * expected = bytes[i], n_good = bytes[i] - n_undef. */
#define OR_ARG_READ 1u
#define OR_ARG_WRITE 2u
int or_check_kernel_args(or_state *s, const uint64_t *ptr, const uint64_t *bytes,
                         const uint32_t *access, uint64_t nargs, or_report *reps);

uint64_t or_emit_records(const or_report *reps, const uint32_t *kind,
                         const uint64_t *dst, const uint64_t *src,
                         const uint64_t *n, uint64_t nreq, int strict,
                         or_record *out, uint64_t cap);

/* Concurrent-access races of a served trace (Sec. 2 itemize: concurrent
 * accesses when several threads are used), requests given in seq order:
 * race_seq[r] = the smallest q < r such that client[q] != client[r],
 * done_ns[q] > submit_ns[r], both copies moved data (moved[q], moved[r]:
 * their device ranges were valid) and one writes what the other reads or
 * writes; -1 if none.  Returns the number of flagged requests. */
uint64_t or_races(const uint32_t *kind, const uint64_t *dst, const uint64_t *src,
                  const uint64_t *n, const uint32_t *client, const uint64_t *submit_ns,
                  const uint64_t *done_ns, const uint8_t *moved, uint64_t count,
                  int64_t *race_seq);

/* state read-back */
int or_read_host_v(const or_state *s, uint64_t off, uint64_t n, uint8_t *out);
int or_read_dev_v(const or_state *s, uint64_t dptr, uint64_t n, uint8_t *out);
uint64_t or_live_count(const or_state *s);

#ifdef __cplusplus
}
#endif
#endif

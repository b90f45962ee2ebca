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
int or_free(or_state *s, uint64_t base, uint32_t *verdict);
int or_mark(or_state *s, uint64_t dptr, uint64_t n, uint8_t value);

int or_check_copy(or_state *s, uint32_t kind, uint64_t dst, uint64_t src,
                  uint64_t n, or_report *rep);
/* requests in order; the whole batch is rejected if any request is invalid */
int or_check_batch(or_state *s, const uint32_t *kind, const uint64_t *dst,
                   const uint64_t *src, const uint64_t *n, uint64_t nreq,
                   or_report *reps, uint64_t *bad_index);

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

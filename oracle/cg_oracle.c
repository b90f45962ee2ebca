/*
 * cg_oracle.c -- plain, byte-by-byte CPU checker (see cg_oracle.h).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * benchmark's CPU-baseline leg, never by the product path.  No code is shared
 * with the GPU library.
 *
 * Every rule below is the plain definition of a check the paper names:
 *   Sec. 2 itemize: copies into or from unallocated device memory; undefined
 *     host data copied to the device; copies larger than the allocation.
 *   Listing 5: the overrun report carries the expected byte count (the copy
 *     size) and the bytes actually found in the allocation.
 *   Sec. 1.1: Memcheck's shadow is bit-precise (A = addressable, V = defined).
 *   Sec. 5: definedness is tracked through host/device, device/host and
 *     device/device transfers, i.e. the V shadow moves with the data.
 * Where the paper is silent the readings are fixed as follows (the GPU
 * library implements the same readings):
 *   R1  A bit of host byte p is bit (p & 7) of byte a[p >> 3]; 1 = addressable.
 *   R2  V byte != 0 means the byte is (partly) undefined; carries copy V
 *       masks exactly.
 *   R3  an unaddressable byte counts only as UNADDR, whatever its V.
 *   R4  offsets are relative to the copy start; -1 when there is none.
 *   R5  device->host / device->device: undefined device-source bytes are
 *       counted as UNDEF and raise a warning (an error in strict mode); the
 *       device source V is only read when the source range is valid.
 *   R6  a new allocation's shadow is all undefined (0xFF).
 *   R7  a copy may start inside an allocation but must end inside the same
 *       allocation; adjacent allocations never combine.
 *   R8  found = bytes from the pointer to its allocation's end; 0 when no
 *       live allocation contains the pointer.
 *   R9  n == 0 is a no-op: no device check, no carry.
 *   R11 host checks run even when a device range fails; the carry does not.
 *   R12 an overlapping device->device copy carries with memmove semantics
 *       and raises a warning.
 *   R13 free: live base -> ok; inside a live allocation -> interior; a freed
 *       base not reused since -> double free; anything else -> unknown.
 *   R14 registering an allocation that overlaps a live one is refused.
 *   R20 concurrent access (or_races): see cg_oracle.h.
 *   R21 pitched copies: only the copied bytes are classified, in the copy's
 *       row-major order; a linear device side must hold the whole extent
 *       (first to one past the last copied byte) in one allocation; a device
 *       array is keyed by its handle, bounded per dimension, and shadowed
 *       densely in (z, y, x) order.
 *   R22 the overlap warning of a pitched device->device copy is raised when
 *       the two spans intersect (for arrays: the same array, spans in its
 *       dense layout); the carry reads every source byte before writing.
 *   R23 memset: the extent must lie in one allocation; the written bytes
 *       become defined.  Kernel arguments: a read argument's range is
 *       checked as a copy source and its undefined bytes counted (a warning
 *       class); a write argument's as a destination, and the whole range
 *       becomes defined after the launch; every read sees the state before
 *       the launch; a zero extent checks only that the pointer lies in a
 *       live allocation.
 */
#include "cg_oracle.h"

#include <stdlib.h>
#include <string.h>

typedef struct {
  uint64_t base;
  uint64_t size;
  uint8_t *shadow; /* NULL: never written, every byte reads 0xFF (R6) */
} live_alloc;

/* Device arrays (Fig. 2: the context's second list) are keyed by handle, a
 * namespace of their own.  Their shadow is dense and row-major (R21): byte
 * (x, y, z) of a W x H x D array (x in bytes) is shadow[(z*H + y)*W + x]. */
typedef struct live_array_s {
  uint64_t handle, w, h, d;
  uint8_t *shadow; /* NULL: never written, reads 0xFF (R6) */
} live_array;

struct or_state {
  uint64_t host_n;
  uint8_t *a_bits;
  uint8_t *host_v;
  int carry;
  int strict;
  live_alloc *live; /* sorted by base, pairwise disjoint */
  uint64_t n_live, cap_live;
  uint64_t *freed; /* sorted freed bases */
  uint64_t n_freed, cap_freed;
  live_array *arrays; /* device arrays, unordered */
  uint64_t n_arrays, cap_arrays;
  uint64_t *freed_arrays; /* handles of destroyed arrays */
  uint64_t n_freed_arrays, cap_freed_arrays;
};

/* ---------------------------------------------------------------- state */

or_state *or_create(uint64_t host_n, const uint8_t *a_bits, const uint8_t *v,
                    int carry, int strict) {
  or_state *s = (or_state *)calloc(1, sizeof *s);
  if (!s) return NULL;
  uint64_t a_len = (host_n + 7) / 8;
  s->host_n = host_n;
  s->a_bits = (uint8_t *)malloc(a_len ? a_len : 1);
  s->host_v = (uint8_t *)malloc(host_n ? host_n : 1);
  if (!s->a_bits || !s->host_v) {
    or_destroy(s);
    return NULL;
  }
  if (a_len) memcpy(s->a_bits, a_bits, a_len);
  if (host_n) memcpy(s->host_v, v, host_n);
  s->carry = carry;
  s->strict = strict;
  return s;
}

void or_destroy(or_state *s) {
  if (!s) return;
  for (uint64_t j = 0; j < s->n_live; j++) free(s->live[j].shadow);
  free(s->live);
  for (uint64_t j = 0; j < s->n_arrays; j++) free(s->arrays[j].shadow);
  free(s->arrays);
  free(s->freed_arrays);
  free(s->freed);
  free(s->a_bits);
  free(s->host_v);
  free(s);
}

uint64_t or_live_count(const or_state *s) { return s->n_live; }

/* index of the first live allocation whose base is > addr */
static uint64_t upper_bound_base(const or_state *s, uint64_t addr) {
  uint64_t lo = 0, hi = s->n_live;
  while (lo < hi) {
    uint64_t mid = lo + (hi - lo) / 2;
    if (s->live[mid].base <= addr)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

/* the live allocation containing addr, or NULL */
static live_alloc *find_alloc(const or_state *s, uint64_t addr) {
  uint64_t ub = upper_bound_base(s, addr);
  if (ub == 0) return NULL;
  live_alloc *a = &s->live[ub - 1];
  if (addr - a->base < a->size) return a;
  return NULL;
}

/* position of the first freed base >= addr */
static uint64_t lower_bound_freed(const or_state *s, uint64_t addr) {
  uint64_t lo = 0, hi = s->n_freed;
  while (lo < hi) {
    uint64_t mid = lo + (hi - lo) / 2;
    if (s->freed[mid] < addr)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

int or_register_alloc(or_state *s, uint64_t base, uint64_t size) {
  if (size == 0) return OR_E_ZERO_SIZE;
  if (base + size < base) return OR_E_WRAP; /* [base, base+size) wraps */
  uint64_t ub = upper_bound_base(s, base);
  /* R14: the predecessor must end at or before base, the successor must
   * start at or after base+size */
  if (ub > 0) {
    live_alloc *p = &s->live[ub - 1];
    if (base - p->base < p->size) return OR_E_OVERLAP;
  }
  if (ub < s->n_live && s->live[ub].base < base + size) return OR_E_OVERLAP;
  if (s->n_live == s->cap_live) {
    uint64_t cap = s->cap_live ? 2 * s->cap_live : 64;
    live_alloc *nl = (live_alloc *)realloc(s->live, cap * sizeof *nl);
    if (!nl) return OR_E_NOMEM;
    s->live = nl;
    s->cap_live = cap;
  }
  memmove(&s->live[ub + 1], &s->live[ub], (s->n_live - ub) * sizeof *s->live);
  s->live[ub].base = base;
  s->live[ub].size = size;
  s->live[ub].shadow = NULL;
  s->n_live++;
  /* R13: freed bases covered by the new allocation are live memory again */
  uint64_t lo = lower_bound_freed(s, base);
  uint64_t hi = lo;
  while (hi < s->n_freed && s->freed[hi] - base < size) hi++;
  if (hi > lo) {
    memmove(&s->freed[lo], &s->freed[hi], (s->n_freed - hi) * sizeof *s->freed);
    s->n_freed -= hi - lo;
  }
  return OR_OK;
}

uint64_t or_register_allocs(or_state *s, const uint64_t *bases, const uint64_t *sizes,
                            uint64_t n, int32_t *status) {
  uint64_t refused = 0;
  for (uint64_t i = 0; i < n; i++) {
    status[i] = or_register_alloc(s, bases[i], sizes[i]);
    if (status[i]) refused++;
  }
  return refused;
}

int or_free(or_state *s, uint64_t base, uint32_t *verdict) {
  if (!verdict) return OR_E_ARG;
  live_alloc *a = find_alloc(s, base);
  if (a && a->base == base) {
    uint64_t j = (uint64_t)(a - s->live);
    free(a->shadow);
    memmove(&s->live[j], &s->live[j + 1], (s->n_live - j - 1) * sizeof *s->live);
    s->n_live--;
    uint64_t pos = lower_bound_freed(s, base);
    if (pos == s->n_freed || s->freed[pos] != base) {
      if (s->n_freed == s->cap_freed) {
        uint64_t cap = s->cap_freed ? 2 * s->cap_freed : 64;
        uint64_t *nf = (uint64_t *)realloc(s->freed, cap * sizeof *nf);
        if (!nf) return OR_E_NOMEM;
        s->freed = nf;
        s->cap_freed = cap;
      }
      memmove(&s->freed[pos + 1], &s->freed[pos], (s->n_freed - pos) * sizeof *s->freed);
      s->freed[pos] = base;
      s->n_freed++;
    }
    *verdict = OR_FREE_OK;
    return OR_OK;
  }
  if (a) {
    *verdict = OR_FREE_INTERIOR;
    return OR_OK;
  }
  uint64_t pos = lower_bound_freed(s, base);
  if (pos < s->n_freed && s->freed[pos] == base)
    *verdict = OR_FREE_DOUBLE;
  else
    *verdict = OR_FREE_UNKNOWN;
  return OR_OK;
}

/* ------------------------------------------------------- shadow access */

static int host_a_bit(const or_state *s, uint64_t pos) {
  return (s->a_bits[pos >> 3] >> (pos & 7)) & 1;
}

static uint8_t dev_v(const live_alloc *a, uint64_t off) {
  return a->shadow ? a->shadow[off] : 0xFF;
}

static int materialise(live_alloc *a) {
  if (a->shadow) return OR_OK;
  a->shadow = (uint8_t *)malloc(a->size);
  if (!a->shadow) return OR_E_NOMEM;
  memset(a->shadow, 0xFF, a->size);
  return OR_OK;
}

int or_mark(or_state *s, uint64_t dptr, uint64_t n, uint8_t value) {
  if (n == 0) return OR_OK;
  live_alloc *a = find_alloc(s, dptr);
  if (!a || n > a->base + a->size - dptr) return OR_E_RANGE;
  int st = materialise(a);
  if (st) return st;
  memset(a->shadow + (dptr - a->base), value, n);
  return OR_OK;
}

int or_read_host_v(const or_state *s, uint64_t off, uint64_t n, uint8_t *out) {
  if (off > s->host_n || n > s->host_n - off) return OR_E_HOST_RANGE;
  if (n) memcpy(out, s->host_v + off, n);
  return OR_OK;
}

int or_read_dev_v(const or_state *s, uint64_t dptr, uint64_t n, uint8_t *out) {
  if (n == 0) return OR_OK;
  live_alloc *a = find_alloc(s, dptr);
  if (!a || n > a->base + a->size - dptr) return OR_E_RANGE;
  for (uint64_t i = 0; i < n; i++) out[i] = dev_v(a, dptr - a->base + i);
  return OR_OK;
}

/* ---------------------------------------------------------------- checks */

/* The device side of a copy (Sec. 2 itemize, Listing 5, R7/R8): returns the
 * containing allocation when [p, p+n) lies wholly inside it, else NULL. */
static live_alloc *device_side(const or_state *s, uint64_t p, uint64_t n,
                               uint64_t *found, uint64_t *abase,
                               uint64_t *asize, uint32_t *flags,
                               uint32_t f_unalloc, uint32_t f_overrun) {
  live_alloc *a = find_alloc(s, p);
  if (!a) {
    *found = 0;
    *abase = 0;
    *asize = 0;
    *flags |= f_unalloc;
    return NULL;
  }
  *found = a->base + a->size - p;
  *abase = a->base;
  *asize = a->size;
  if (n > *found) {
    *flags |= f_overrun;
    return NULL;
  }
  return a;
}

static int validate(const or_state *s, uint32_t kind, uint64_t dst,
                    uint64_t src, uint64_t n) {
  if (kind != OR_HTOD && kind != OR_DTOH && kind != OR_DTOD) return OR_E_KIND;
  if (kind == OR_HTOD || kind == OR_DTOH) {
    uint64_t h = kind == OR_HTOD ? src : dst;
    if (h > s->host_n || n > s->host_n - h) return OR_E_HOST_RANGE;
  }
  return OR_OK;
}

static int check_one(or_state *s, uint32_t kind, uint64_t dst, uint64_t src,
                     uint64_t n, or_report *r) {
  memset(r, 0, sizeof *r);
  r->first_bad_off = -1;
  r->first_unaddr_off = -1;
  r->first_undef_off = -1;
  r->race_seq = -1;
  r->expected = n;
  if (n == 0) return OR_OK; /* R9 */

  live_alloc *da = NULL, *sa = NULL;
  if (kind == OR_HTOD || kind == OR_DTOD)
    da = device_side(s, dst, n, &r->found_dst, &r->alloc_base_dst,
                     &r->alloc_size_dst, &r->flags, OR_F_UNALLOC_DST,
                     OR_F_OVERRUN_DST);
  if (kind == OR_DTOH || kind == OR_DTOD)
    sa = device_side(s, src, n, &r->found_src, &r->alloc_base_src,
                     &r->alloc_size_src, &r->flags, OR_F_UNALLOC_SRC,
                     OR_F_OVERRUN_SRC);

  /* classify every byte (R1-R5) */
  for (uint64_t i = 0; i < n; i++) {
    uint32_t cls = OR_BYTE_GOOD;
    if (kind == OR_HTOD) {
      if (!host_a_bit(s, src + i))
        cls = OR_BYTE_UNADDR;
      else if (s->host_v[src + i] != 0)
        cls = OR_BYTE_UNDEF;
    } else if (kind == OR_DTOH) {
      if (!host_a_bit(s, dst + i))
        cls = OR_BYTE_UNADDR;
      else if (sa && dev_v(sa, src - sa->base + i) != 0)
        cls = OR_BYTE_UNDEF;
    } else {
      if (sa && dev_v(sa, src - sa->base + i) != 0) cls = OR_BYTE_UNDEF;
    }
    if (cls == OR_BYTE_GOOD) {
      r->n_good++;
    } else if (cls == OR_BYTE_UNADDR) {
      r->n_unaddr++;
      if (r->first_unaddr_off < 0) r->first_unaddr_off = (int64_t)i;
    } else {
      r->n_undef++;
      if (r->first_undef_off < 0) r->first_undef_off = (int64_t)i;
    }
    if (cls != OR_BYTE_GOOD && r->first_bad_off < 0) {
      r->first_bad_off = (int64_t)i;
      r->first_bad_kind = cls;
    }
  }
  if (r->n_unaddr) r->flags |= OR_F_HOST_UNADDR;
  if (r->n_undef) r->flags |= kind == OR_HTOD ? OR_F_HOST_UNDEF : OR_F_DEV_UNDEF_SRC;
  if (kind == OR_DTOD) {
    uint64_t dist = src <= dst ? dst - src : src - dst;
    if (dist < n) r->flags |= OR_F_DTOD_OVERLAP;
  }

  /* carry the V shadow with the data (Sec. 5), only over valid ranges (R11) */
  if (!s->carry) return OR_OK;
  if (kind == OR_HTOD && da) {
    int st = materialise(da);
    if (st) return st;
    uint64_t o = dst - da->base;
    for (uint64_t i = 0; i < n; i++)
      da->shadow[o + i] = host_a_bit(s, src + i) ? s->host_v[src + i] : 0xFF;
  } else if (kind == OR_DTOH && sa) {
    uint64_t o = src - sa->base;
    for (uint64_t i = 0; i < n; i++)
      if (host_a_bit(s, dst + i)) s->host_v[dst + i] = dev_v(sa, o + i);
  } else if (kind == OR_DTOD && sa && da) {
    uint8_t *tmp = (uint8_t *)malloc(n); /* R12: read everything first */
    if (!tmp) return OR_E_NOMEM;
    uint64_t os = src - sa->base;
    for (uint64_t i = 0; i < n; i++) tmp[i] = dev_v(sa, os + i);
    int st = materialise(da);
    if (st) {
      free(tmp);
      return st;
    }
    uint64_t od = dst - da->base;
    for (uint64_t i = 0; i < n; i++) da->shadow[od + i] = tmp[i];
    free(tmp);
  }
  return OR_OK;
}

int or_check_copy(or_state *s, uint32_t kind, uint64_t dst, uint64_t src,
                  uint64_t n, or_report *rep) {
  if (!s || !rep) return OR_E_ARG;
  int st = validate(s, kind, dst, src, n);
  if (st) return st;
  return check_one(s, kind, dst, src, n, rep);
}

int or_check_batch(or_state *s, const uint32_t *kind, const uint64_t *dst,
                   const uint64_t *src, const uint64_t *n, uint64_t nreq,
                   or_report *reps, uint64_t *bad_index) {
  if (!s || (nreq && (!kind || !dst || !src || !n || !reps))) return OR_E_ARG;
  for (uint64_t i = 0; i < nreq; i++) {
    int st = validate(s, kind[i], dst[i], src[i], n[i]);
    if (st) {
      if (bad_index) *bad_index = i;
      return st;
    }
  }
  for (uint64_t i = 0; i < nreq; i++) {
    int st = check_one(s, kind[i], dst[i], src[i], n[i], &reps[i]);
    if (st) {
      if (bad_index) *bad_index = i;
      return st;
    }
  }
  return OR_OK;
}

/* ------------------------------------------- pitched copies, arrays */

static live_array *find_array(const or_state *s, uint64_t handle) {
  for (uint64_t j = 0; j < s->n_arrays; j++)
    if (s->arrays[j].handle == handle) return &s->arrays[j];
  return NULL;
}

static int handle_freed(const or_state *s, uint64_t handle) {
  for (uint64_t j = 0; j < s->n_freed_arrays; j++)
    if (s->freed_arrays[j] == handle) return 1;
  return 0;
}

int or_register_array(or_state *s, uint64_t handle, uint64_t w, uint64_t h, uint64_t d) {
  if (!s) return OR_E_ARG;
  if (w == 0 || h == 0 || d == 0) return OR_E_ZERO_SIZE;
  if (h > UINT64_MAX / w || d > UINT64_MAX / (w * h)) return OR_E_WRAP;
  if (find_array(s, handle)) return OR_E_OVERLAP;
  if (s->n_arrays == s->cap_arrays) {
    uint64_t cap = s->cap_arrays ? 2 * s->cap_arrays : 8;
    live_array *p = (live_array *)realloc(s->arrays, cap * sizeof *p);
    if (!p) return OR_E_NOMEM;
    s->arrays = p;
    s->cap_arrays = cap;
  }
  live_array *a = &s->arrays[s->n_arrays++];
  a->handle = handle;
  a->w = w;
  a->h = h;
  a->d = d;
  a->shadow = NULL;
  /* a re-used handle is no longer "freed" */
  for (uint64_t j = 0; j < s->n_freed_arrays; j++)
    if (s->freed_arrays[j] == handle) s->freed_arrays[j] = s->freed_arrays[--s->n_freed_arrays];
  return OR_OK;
}

int or_free_array(or_state *s, uint64_t handle, uint32_t *verdict) {
  if (!s || !verdict) return OR_E_ARG;
  live_array *a = find_array(s, handle);
  if (a) {
    free(a->shadow);
    *a = s->arrays[--s->n_arrays];
    if (s->n_freed_arrays == s->cap_freed_arrays) {
      uint64_t cap = s->cap_freed_arrays ? 2 * s->cap_freed_arrays : 8;
      uint64_t *p = (uint64_t *)realloc(s->freed_arrays, cap * sizeof *p);
      if (!p) return OR_E_NOMEM;
      s->freed_arrays = p;
      s->cap_freed_arrays = cap;
    }
    s->freed_arrays[s->n_freed_arrays++] = handle;
    *verdict = OR_FREE_OK;
  } else {
    *verdict = handle_freed(s, handle) ? OR_FREE_DOUBLE : OR_FREE_UNKNOWN;
  }
  return OR_OK;
}

int or_read_array_v(const or_state *s, uint64_t handle, uint64_t off, uint64_t n, uint8_t *out) {
  live_array *a = find_array(s, handle);
  if (!a) return OR_E_RANGE;
  const uint64_t total = a->w * a->h * a->d;
  if (off > total || n > total - off) return OR_E_RANGE;
  for (uint64_t i = 0; i < n; i++) out[i] = a->shadow ? a->shadow[off + i] : 0xFF;
  return OR_OK;
}

/* One side of a 3-D copy as the checks see it. */
typedef struct {
  int array;          /* 1: a device array, 0: linear memory / host image */
  live_alloc *alloc;  /* linear device side, valid range: its allocation */
  live_array *arr;    /* array side, valid range: the array */
  uint64_t start;     /* linear: address (host offset) of copy byte (0,0,0) */
  uint64_t pitch;     /* bytes between rows */
  uint64_t slice;     /* bytes between slices */
  int ok;             /* the range check passed */
} side3d;

/* Byte (i, y, z) of the copy (x-in-bytes, row, slice, all relative to the
 * copy's origin) on one side: a host offset, a device address, or an index
 * into an array's dense shadow. */
static uint64_t side_pos(const side3d *sd, uint64_t i, uint64_t y, uint64_t z) {
  return sd->start + z * sd->slice + y * sd->pitch + i;
}

static uint8_t side_dev_v(const side3d *sd, uint64_t pos) {
  if (sd->array) return sd->arr->shadow ? sd->arr->shadow[pos] : 0xFF;
  return dev_v(sd->alloc, pos - sd->alloc->base);
}

static int side_materialise(side3d *sd) {
  if (!sd->array) return materialise(sd->alloc);
  if (sd->arr->shadow) return OR_OK;
  const uint64_t total = sd->arr->w * sd->arr->h * sd->arr->d;
  sd->arr->shadow = (uint8_t *)malloc(total);
  if (!sd->arr->shadow) return OR_E_NOMEM;
  memset(sd->arr->shadow, 0xFF, total);
  return OR_OK;
}

static uint8_t *side_dev_byte(side3d *sd, uint64_t pos) {
  if (sd->array) return &sd->arr->shadow[pos];
  return &sd->alloc->shadow[pos - sd->alloc->base];
}

/* start = origin address, extent = bytes from the first to one past the last
 * copied byte; returns OR_E_WRAP if either does not fit in 64 bits. */
static int linear_geometry(const or_side3d *q, uint64_t w, uint64_t h, uint64_t d,
                           uint64_t *start, uint64_t *extent, uint64_t *pitch, uint64_t *slice) {
  const uint64_t p = q->pitch, rows = q->rows;
  if (rows && p > UINT64_MAX / rows) return OR_E_WRAP;
  const uint64_t sl = p * rows;
  if ((q->z && sl && q->z > UINT64_MAX / sl) || (q->y && p && q->y > UINT64_MAX / p))
    return OR_E_WRAP;
  const uint64_t o1 = q->z * sl, o2 = q->y * p;
  if (o1 > UINT64_MAX - o2 || o1 + o2 > UINT64_MAX - q->x) return OR_E_WRAP;
  const uint64_t off = o1 + o2 + q->x;
  if (q->ptr > UINT64_MAX - off) return OR_E_WRAP;
  if ((d - 1) && sl && d - 1 > UINT64_MAX / sl) return OR_E_WRAP;
  if ((h - 1) && p && h - 1 > UINT64_MAX / p) return OR_E_WRAP;
  const uint64_t e1 = (d - 1) * sl, e2 = (h - 1) * p;
  if (e1 > UINT64_MAX - e2 || e1 + e2 > UINT64_MAX - w) return OR_E_WRAP;
  *start = q->ptr + off;
  *extent = e1 + e2 + w;
  *pitch = p;
  *slice = sl;
  return OR_OK;
}

static int check_side_args(const or_side3d *q, uint64_t w, uint64_t h, uint64_t d) {
  if (q->reserved) return OR_E_ARG;
  if (q->is_array) return OR_OK;
  if ((h > 1 || d > 1) && q->pitch < w) return OR_E_ARG;
  if (d > 1 && q->rows < h) return OR_E_ARG;
  return OR_OK;
}

/* The device side of a 3-D copy: array lookup by handle with a bound per
 * dimension, or the linear range check over the extent. */
static int device_side3d(or_state *s, const or_side3d *q, uint64_t w, uint64_t h, uint64_t d,
                         side3d *sd, uint64_t *found, uint64_t *abase, uint64_t *asize,
                         uint32_t *flags, uint32_t f_unalloc, uint32_t f_overrun) {
  memset(sd, 0, sizeof *sd);
  if (q->is_array) {
    sd->array = 1;
    live_array *a = find_array(s, q->ptr);
    *found = *abase = *asize = 0;
    if (!a) {
      *flags |= f_unalloc;
      return OR_OK;
    }
    sd->arr = a;
    *abase = a->handle;
    *asize = a->w * a->h * a->d;
    const int inside = q->x < a->w && q->y < a->h && q->z < a->d;
    if (inside) *found = *asize - ((q->z * a->h + q->y) * a->w + q->x);
    /* per dimension: origin + extent within the array's box (no overflow:
     * each origin is compared before adding) */
    const int fits = q->x <= a->w && w <= a->w - q->x && q->y <= a->h && h <= a->h - q->y &&
                     q->z <= a->d && d <= a->d - q->z;
    if (!fits) {
      *flags |= f_overrun;
      return OR_OK;
    }
    sd->start = (q->z * a->h + q->y) * a->w + q->x;
    sd->pitch = a->w;
    sd->slice = a->w * a->h;
    sd->ok = 1;
    return OR_OK;
  }
  uint64_t start, ext;
  int st = linear_geometry(q, w, h, d, &start, &ext, &sd->pitch, &sd->slice);
  if (st) return st;
  sd->start = start;
  sd->alloc = device_side(s, start, ext, found, abase, asize, flags, f_unalloc, f_overrun);
  sd->ok = sd->alloc != NULL;
  return OR_OK;
}

int or_check_copy3d(or_state *s, const or_copy3d *q, or_report *r) {
  if (!s || !q || !r) return OR_E_ARG;
  const uint32_t kind = q->kind;
  if (kind != OR_HTOD && kind != OR_DTOH && kind != OR_DTOD) return OR_E_KIND;
  if (q->reserved || q->dst.reserved || q->src.reserved) return OR_E_ARG;
  const uint64_t w = q->width, h = q->height, d = q->depth;
  if (w && h && (h > UINT64_MAX / w || (d && d > UINT64_MAX / (w * h)))) return OR_E_WRAP;
  const uint64_t n = w * h * d;
  /* the host side is the bound image, never an array */
  if ((kind == OR_HTOD && q->src.is_array) || (kind == OR_DTOH && q->dst.is_array))
    return OR_E_ARG;
  memset(r, 0, sizeof *r);
  r->first_bad_off = -1;
  r->first_unaddr_off = -1;
  r->first_undef_off = -1;
  r->race_seq = -1;
  r->expected = n;
  if (n == 0) return OR_OK; /* R9 */
  int st = check_side_args(&q->dst, w, h, d);
  if (!st) st = check_side_args(&q->src, w, h, d);
  if (st) return st;
  side3d host, ds, ss;
  memset(&host, 0, sizeof host);
  memset(&ds, 0, sizeof ds);
  memset(&ss, 0, sizeof ss);
  if (kind == OR_HTOD || kind == OR_DTOH) {
    const or_side3d *hq = kind == OR_HTOD ? &q->src : &q->dst;
    uint64_t ext;
    st = linear_geometry(hq, w, h, d, &host.start, &ext, &host.pitch, &host.slice);
    if (st) return st;
    if (host.start > s->host_n || ext > s->host_n - host.start) return OR_E_HOST_RANGE;
  }
  if (kind == OR_HTOD || kind == OR_DTOD) {
    st = device_side3d(s, &q->dst, w, h, d, &ds, &r->found_dst, &r->alloc_base_dst,
                       &r->alloc_size_dst, &r->flags, OR_F_UNALLOC_DST, OR_F_OVERRUN_DST);
    if (st) return st;
  }
  if (kind == OR_DTOH || kind == OR_DTOD) {
    st = device_side3d(s, &q->src, w, h, d, &ss, &r->found_src, &r->alloc_base_src,
                       &r->alloc_size_src, &r->flags, OR_F_UNALLOC_SRC, OR_F_OVERRUN_SRC);
    if (st) return st;
  }
  /* classification in the copy's own row-major order */
  for (uint64_t z = 0; z < d; z++)
    for (uint64_t y = 0; y < h; y++)
      for (uint64_t i = 0; i < w; i++) {
        const uint64_t o = (z * h + y) * w + i; /* linear offset */
        uint32_t cls = OR_BYTE_GOOD;
        if (kind == OR_HTOD) {
          const uint64_t hp = side_pos(&host, i, y, z);
          if (!host_a_bit(s, hp))
            cls = OR_BYTE_UNADDR;
          else if (s->host_v[hp] != 0)
            cls = OR_BYTE_UNDEF;
        } else if (kind == OR_DTOH) {
          if (!host_a_bit(s, side_pos(&host, i, y, z)))
            cls = OR_BYTE_UNADDR;
          else if (ss.ok && side_dev_v(&ss, side_pos(&ss, i, y, z)) != 0)
            cls = OR_BYTE_UNDEF;
        } else if (ss.ok && side_dev_v(&ss, side_pos(&ss, i, y, z)) != 0) {
          cls = OR_BYTE_UNDEF;
        }
        if (cls == OR_BYTE_GOOD) {
          r->n_good++;
          continue;
        }
        if (cls == OR_BYTE_UNADDR) {
          r->n_unaddr++;
          if (r->first_unaddr_off < 0) r->first_unaddr_off = (int64_t)o;
        } else {
          r->n_undef++;
          if (r->first_undef_off < 0) r->first_undef_off = (int64_t)o;
        }
        if (r->first_bad_off < 0) {
          r->first_bad_off = (int64_t)o;
          r->first_bad_kind = cls;
        }
      }
  if (r->n_unaddr) r->flags |= OR_F_HOST_UNADDR;
  if (r->n_undef) r->flags |= kind == OR_HTOD ? OR_F_HOST_UNDEF : OR_F_DEV_UNDEF_SRC;
  /* overlap warning (R22): the two spans, first to one past the last copied
   * byte, intersect (arrays: the same array, spans in its dense layout) */
  if (kind == OR_DTOD && q->dst.is_array == q->src.is_array) {
    const int same = q->dst.is_array ? q->dst.ptr == q->src.ptr : 1;
    if (same) {
      uint64_t dstart, dext, sstart, sext, p0, s0;
      if (q->dst.is_array) {
        live_array *a = find_array(s, q->dst.ptr);
        if (a) {
          dstart = (q->dst.z * a->h + q->dst.y) * a->w + q->dst.x;
          sstart = (q->src.z * a->h + q->src.y) * a->w + q->src.x;
          dext = sext = ((d - 1) * a->h + (h - 1)) * a->w + w;
          if (dstart < sstart + sext && sstart < dstart + dext) r->flags |= OR_F_DTOD_OVERLAP;
        }
      } else if (!linear_geometry(&q->dst, w, h, d, &dstart, &dext, &p0, &s0) &&
                 !linear_geometry(&q->src, w, h, d, &sstart, &sext, &p0, &s0)) {
        if (dstart - sstart < sext || sstart - dstart < dext) r->flags |= OR_F_DTOD_OVERLAP;
      }
    }
  }
  if (!s->carry) return OR_OK;
  /* R11: no carry unless every device side passed its range check */
  if (kind == OR_HTOD && ds.ok) {
    if ((st = side_materialise(&ds))) return st;
    for (uint64_t z = 0; z < d; z++)
      for (uint64_t y = 0; y < h; y++)
        for (uint64_t i = 0; i < w; i++) {
          const uint64_t hp = side_pos(&host, i, y, z);
          *side_dev_byte(&ds, side_pos(&ds, i, y, z)) = host_a_bit(s, hp) ? s->host_v[hp] : 0xFF;
        }
  } else if (kind == OR_DTOH && ss.ok) {
    for (uint64_t z = 0; z < d; z++)
      for (uint64_t y = 0; y < h; y++)
        for (uint64_t i = 0; i < w; i++) {
          const uint64_t hp = side_pos(&host, i, y, z);
          if (host_a_bit(s, hp)) s->host_v[hp] = side_dev_v(&ss, side_pos(&ss, i, y, z));
        }
  } else if (kind == OR_DTOD && ss.ok && ds.ok) {
    uint8_t *tmp = (uint8_t *)malloc(n); /* every source byte before any write */
    if (!tmp) return OR_E_NOMEM;
    for (uint64_t z = 0; z < d; z++)
      for (uint64_t y = 0; y < h; y++)
        for (uint64_t i = 0; i < w; i++)
          tmp[(z * h + y) * w + i] = side_dev_v(&ss, side_pos(&ss, i, y, z));
    if ((st = side_materialise(&ds))) {
      free(tmp);
      return st;
    }
    for (uint64_t z = 0; z < d; z++)
      for (uint64_t y = 0; y < h; y++)
        for (uint64_t i = 0; i < w; i++)
          *side_dev_byte(&ds, side_pos(&ds, i, y, z)) = tmp[(z * h + y) * w + i];
    free(tmp);
  }
  return OR_OK;
}

/* ------------------------------------- memset and kernel arguments */

static void blank_report(or_report *r, uint64_t n) {
  memset(r, 0, sizeof *r);
  r->first_bad_off = -1;
  r->first_unaddr_off = -1;
  r->first_undef_off = -1;
  r->race_seq = -1;
  r->expected = n;
}

int or_memset(or_state *s, uint64_t dptr, uint64_t pitch, uint64_t width, uint64_t height,
              or_report *r) {
  if (!s || !r) return OR_E_ARG;
  if (height > 1 && pitch < width) return OR_E_ARG;
  if (width && height > UINT64_MAX / width) return OR_E_WRAP;
  const uint64_t n = width * height;
  blank_report(r, n);
  if (n == 0) return OR_OK; /* R9 */
  if (height - 1 > (UINT64_MAX - width) / (pitch ? pitch : 1)) return OR_E_WRAP;
  const uint64_t ext = (height - 1) * pitch + width;
  live_alloc *a = device_side(s, dptr, ext, &r->found_dst, &r->alloc_base_dst,
                              &r->alloc_size_dst, &r->flags, OR_F_UNALLOC_DST, OR_F_OVERRUN_DST);
  r->n_good = n; /* nothing is read: no byte can be bad */
  if (!a || !s->carry) return OR_OK;
  int st = materialise(a);
  if (st) return st;
  for (uint64_t y = 0; y < height; y++)
    for (uint64_t i = 0; i < width; i++) a->shadow[dptr + y * pitch + i - a->base] = 0x00;
  return OR_OK;
}

int or_check_kernel_args(or_state *s, const uint64_t *ptr, const uint64_t *bytes,
                         const uint32_t *access, uint64_t nargs, or_report *reps) {
  if (!s || (nargs && (!ptr || !bytes || !access || !reps))) return OR_E_ARG;
  for (uint64_t i = 0; i < nargs; i++)
    if (access[i] == 0 || (access[i] & ~(OR_ARG_READ | OR_ARG_WRITE))) return OR_E_ARG;
  /* every read sees the state before the launch */
  for (uint64_t i = 0; i < nargs; i++) {
    or_report *r = &reps[i];
    blank_report(r, bytes[i]);
    live_alloc *ra = NULL;
    if (access[i] & OR_ARG_READ)
      ra = device_side(s, ptr[i], bytes[i], &r->found_src, &r->alloc_base_src,
                       &r->alloc_size_src, &r->flags, OR_F_UNALLOC_SRC, OR_F_OVERRUN_SRC);
    if (access[i] & OR_ARG_WRITE)
      (void)device_side(s, ptr[i], bytes[i], &r->found_dst, &r->alloc_base_dst,
                        &r->alloc_size_dst, &r->flags, OR_F_UNALLOC_DST, OR_F_OVERRUN_DST);
    for (uint64_t k = 0; ra && k < bytes[i]; k++) {
      if (dev_v(ra, ptr[i] + k - ra->base) == 0) continue;
      r->n_undef++;
      if (r->first_undef_off < 0) {
        r->first_undef_off = (int64_t)k;
        r->first_bad_off = (int64_t)k;
        r->first_bad_kind = OR_BYTE_UNDEF;
      }
    }
    r->n_good = bytes[i] - r->n_undef;
    if (r->n_undef) r->flags |= OR_F_DEV_UNDEF_SRC;
  }
  if (!s->carry) return OR_OK;
  /* then every written argument whose range is valid becomes defined */
  for (uint64_t i = 0; i < nargs; i++) {
    if (!(access[i] & OR_ARG_WRITE) || bytes[i] == 0) continue;
    if (reps[i].flags & (OR_F_UNALLOC_DST | OR_F_OVERRUN_DST)) continue;
    live_alloc *a = find_alloc(s, ptr[i]);
    int st = materialise(a);
    if (st) return st;
    memset(a->shadow + (ptr[i] - a->base), 0x00, bytes[i]);
  }
  return OR_OK;
}

/* One record per set flag, in (request, flag bit) order. */
uint64_t or_emit_records(const or_report *reps, const uint32_t *kind,
                         const uint64_t *dst, const uint64_t *src,
                         const uint64_t *n, uint64_t nreq, int strict,
                         or_record *out, uint64_t cap) {
  uint64_t k = 0;
  for (uint64_t i = 0; i < nreq; i++) {
    const or_report *r = &reps[i];
    for (uint32_t b = 0; b < OR_NFLAGS; b++) {
      uint32_t f = 1u << b;
      if (!(r->flags & f)) continue;
      or_record rec;
      memset(&rec, 0, sizeof rec);
      rec.req = i;
      rec.cls = b;
      rec.expected = n[i];
      rec.severity = 0;
      if (f == OR_F_UNALLOC_DST || f == OR_F_UNALLOC_SRC) {
        rec.off = 0;
        rec.count = n[i];
        rec.found = 0;
      } else if (f == OR_F_OVERRUN_DST || f == OR_F_OVERRUN_SRC) {
        uint64_t found = f == OR_F_OVERRUN_DST ? r->found_dst : r->found_src;
        rec.off = (int64_t)found;
        rec.count = n[i] - found;
        rec.found = found;
      } else if (f == OR_F_HOST_UNADDR) {
        rec.off = r->first_unaddr_off;
        rec.count = r->n_unaddr;
        rec.found = n[i] - r->n_unaddr;
      } else if (f == OR_F_HOST_UNDEF || f == OR_F_DEV_UNDEF_SRC) {
        rec.off = r->first_undef_off;
        rec.count = r->n_undef;
        rec.found = r->n_good;
        if (f == OR_F_DEV_UNDEF_SRC && !strict) rec.severity = 1;
      } else if (f == OR_F_DTOD_OVERLAP) {
        uint64_t dist = src[i] <= dst[i] ? dst[i] - src[i] : src[i] - dst[i];
        rec.off = (int64_t)(dst[i] - src[i]);
        rec.count = n[i] - dist;
        rec.found = 0;
        rec.severity = 1;
        (void)kind;
      } else { /* OR_F_CONCURRENT */
        rec.off = r->race_seq;
        rec.count = n[i];
        rec.found = 0;
        rec.severity = 1;
      }
      if (k < cap) out[k] = rec;
      k++;
    }
  }
  return k;
}

/* ------------------------------------------------------------- races */

/* [a, a+na) and [b, b+nb) share a byte */
static int meets(uint64_t a, uint64_t na, uint64_t b, uint64_t nb) {
  return a < b + nb && b < a + na;
}

/* Which address space each side of a copy lives in: 0 host, 1 device. */
static int dst_space(uint32_t kind) { return kind == OR_DTOH ? 0 : 1; }
static int src_space(uint32_t kind) { return kind == OR_HTOD ? 0 : 1; }

uint64_t or_races(const uint32_t *kind, const uint64_t *dst, const uint64_t *src,
                  const uint64_t *n, const uint32_t *client, const uint64_t *submit_ns,
                  const uint64_t *done_ns, const uint8_t *moved, uint64_t count,
                  int64_t *race_seq) {
  uint64_t flagged = 0;
  for (uint64_t r = 0; r < count; r++) {
    race_seq[r] = -1;
    if (!moved[r] || n[r] == 0) continue;
    for (uint64_t q = 0; q < r; q++) {
      if (!moved[q] || n[q] == 0 || client[q] == client[r]) continue;
      if (!(done_ns[q] > submit_ns[r])) continue; /* q finished before r was sent */
      /* q writes what r reads, q writes what r writes, q reads what r writes */
      int hit = 0;
      if (dst_space(kind[q]) == src_space(kind[r]) && meets(dst[q], n[q], src[r], n[r])) hit = 1;
      if (dst_space(kind[q]) == dst_space(kind[r]) && meets(dst[q], n[q], dst[r], n[r])) hit = 1;
      if (src_space(kind[q]) == dst_space(kind[r]) && meets(src[q], n[q], dst[r], n[r])) hit = 1;
      if (hit) {
        race_seq[r] = (int64_t)q;
        flagged++;
        break;
      }
    }
  }
  return flagged;
}

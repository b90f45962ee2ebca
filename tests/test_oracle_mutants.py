"""Plant plausible mistakes in a copy of the CPU oracle and check that the
pins catch every one of them (a pin suite that a dropped term, a flipped
comparison or a wrong index can pass would not pin anything).

Each mutant is compiled from the oracle source with one textual change and
run through ``tests/pins.py`` in a child process, so that a mutant that
crashes counts as caught without taking the test run down.
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402

SRC = open(os.path.join(ROOT, "oracle", "cg_oracle.c")).read()

MUTANTS = {
    "a_bit_msb_first": ("return (s->a_bits[pos >> 3] >> (pos & 7)) & 1;",
                        "return (s->a_bits[pos >> 3] >> (7 - (pos & 7))) & 1;"),
    "a_bit_no_offset": ("if (!host_a_bit(s, src + i))", "if (!host_a_bit(s, i))"),
    "undef_only_full_mask": ("else if (s->host_v[src + i] != 0)",
                             "else if (s->host_v[src + i] == 0xFF)"),
    "undef_before_unaddr": (
        "      if (!host_a_bit(s, src + i))\n        cls = OR_BYTE_UNADDR;\n"
        "      else if (s->host_v[src + i] != 0)\n        cls = OR_BYTE_UNDEF;",
        "      if (s->host_v[src + i] != 0)\n        cls = OR_BYTE_UNDEF;\n"
        "      else if (!host_a_bit(s, src + i))\n        cls = OR_BYTE_UNADDR;"),
    "dtoh_ignores_dest_a": ("if (!host_a_bit(s, dst + i))\n        cls = OR_BYTE_UNADDR;",
                            "if (0)\n        cls = OR_BYTE_UNADDR;"),
    "last_unaddr_not_first": ("if (r->first_unaddr_off < 0) r->first_unaddr_off = (int64_t)i;",
                              "r->first_unaddr_off = (int64_t)i;"),
    "first_bad_kind_unset": ("r->first_bad_off = (int64_t)i;\n      r->first_bad_kind = cls;",
                             "r->first_bad_off = (int64_t)i;\n      r->first_bad_kind = OR_BYTE_UNDEF;"),
    "p3_first_bad_kind_unset": ("r->first_bad_off = (int64_t)o;\n          r->first_bad_kind = cls;",
                                "r->first_bad_off = (int64_t)o;\n          r->first_bad_kind = OR_BYTE_UNDEF;"),
    "good_count_dropped": ("      r->n_good++;\n    } else", "      ;\n    } else"),
    "p3_good_count_dropped": ("          r->n_good++;\n          continue;", "          continue;"),
    "overrun_off_by_one": ("if (n > *found) {", "if (n >= *found) {"),
    "found_off_by_one": ("*found = a->base + a->size - p;", "*found = a->base + a->size - p - 1;"),
    "containment_inclusive": ("if (addr - a->base < a->size) return a;",
                              "if (addr - a->base <= a->size) return a;"),
    "lookup_first_not_last": ("  live_alloc *a = &s->live[ub - 1];",
                              "  live_alloc *a = &s->live[0];"),
    "fresh_shadow_defined": ("return a->shadow ? a->shadow[off] : 0xFF;",
                             "return a->shadow ? a->shadow[off] : 0x00;"),
    "htod_carry_ignores_a": (
        "da->shadow[o + i] = host_a_bit(s, src + i) ? s->host_v[src + i] : 0xFF;",
        "da->shadow[o + i] = s->host_v[src + i];"),
    "dtoh_carry_ignores_a": ("if (host_a_bit(s, dst + i)) s->host_v[dst + i] = dev_v(sa, o + i);",
                             "s->host_v[dst + i] = dev_v(sa, o + i);"),
    "carry_on_overrun": ("if (kind == OR_HTOD && da) {", "if (kind == OR_HTOD && r->alloc_size_dst) {\n"
                         "    if (!da) da = find_alloc(s, dst);"),
    "dtod_forward_copy": ("for (uint64_t i = 0; i < n; i++) da->shadow[od + i] = tmp[i];",
                          "for (uint64_t i = 0; i < n; i++) da->shadow[od + i] = dev_v(sa, os + i);"),
    "overlap_inclusive": ("if (dist < n) r->flags |= OR_F_DTOD_OVERLAP;",
                          "if (dist <= n) r->flags |= OR_F_DTOD_OVERLAP;"),
    "double_free_as_unknown": ("    *verdict = OR_FREE_DOUBLE;", "    *verdict = OR_FREE_UNKNOWN;"),
    "freed_set_never_pruned": ("while (hi < s->n_freed && s->freed[hi] - base < size) hi++;",
                               "(void)size;"),
    "overlap_check_skips_successor": (
        "if (ub < s->n_live && s->live[ub].base < base + size) return OR_E_OVERLAP;", ""),
    "overrun_record_count": ("rec.count = n[i] - found;", "rec.count = found;"),
    "warning_severity_lost": ("if (f == OR_F_DEV_UNDEF_SRC && !strict) rec.severity = 1;", ""),
    "race_same_client_counts": ("if (!moved[q] || n[q] == 0 || client[q] == client[r]) continue;",
                                "if (!moved[q] || n[q] == 0) continue;"),
    "race_ignores_done_time": ("if (!(done_ns[q] > submit_ns[r])) continue; /* q finished before r was sent */",
                               ""),
    "race_reads_conflict": ("if (src_space(kind[q]) == dst_space(kind[r]) && meets(src[q], n[q], dst[r], n[r])) hit = 1;",
                            "if (src_space(kind[q]) == src_space(kind[r]) && meets(src[q], n[q], src[r], n[r])) hit = 1;"),
    # pitched copies and arrays
    "p3_offset_transposed": ("const uint64_t o = (z * h + y) * w + i; /* linear offset */",
                             "const uint64_t o = (y * d + z) * w + i; /* linear offset */"),
    "p3_extent_whole_last_row": ("*extent = e1 + e2 + w;", "*extent = e1 + e2 + p;"),
    "p3_slice_uses_height": ("const uint64_t p = q->pitch, rows = q->rows;",
                             "const uint64_t p = q->pitch, rows = h;"),
    "p3_pitch_check_dropped": ("if ((h > 1 || d > 1) && q->pitch < w) return OR_E_ARG;", ""),
    "p3_array_bound_exclusive": ("w <= a->w - q->x", "w < a->w - q->x"),
    "p3_array_pitch_is_height": ("    sd->pitch = a->w;\n", "    sd->pitch = a->h;\n"),
    "p3_array_found_whole": ("if (inside) *found = *asize - ((q->z * a->h + q->y) * a->w + q->x);",
                             "if (inside) *found = *asize;"),
    "p3_dtod_no_staging": ("*side_dev_byte(&ds, side_pos(&ds, i, y, z)) = tmp[(z * h + y) * w + i];",
                           "*side_dev_byte(&ds, side_pos(&ds, i, y, z)) = side_dev_v(&ss, side_pos(&ss, i, y, z));"),
    "p3_overlap_by_count": ("if (dstart - sstart < sext || sstart - dstart < dext)",
                            "if (dstart - sstart < n || sstart - dstart < n)"),
    "p3_htod_carry_ignores_a": (
        "*side_dev_byte(&ds, side_pos(&ds, i, y, z)) = host_a_bit(s, hp) ? s->host_v[hp] : 0xFF;",
        "*side_dev_byte(&ds, side_pos(&ds, i, y, z)) = s->host_v[hp];"),
    "p3_array_double_destroy_unknown": (
        "*verdict = handle_freed(s, handle) ? OR_FREE_DOUBLE : OR_FREE_UNKNOWN;",
        "*verdict = OR_FREE_UNKNOWN;"),
    "p3_dtoh_carry_ignores_a": (
        "if (host_a_bit(s, hp)) s->host_v[hp] = side_dev_v(&ss, side_pos(&ss, i, y, z));",
        "s->host_v[hp] = side_dev_v(&ss, side_pos(&ss, i, y, z));"),
    "p3_origin_ignores_y": ("const uint64_t o1 = q->z * sl, o2 = q->y * p;",
                            "const uint64_t o1 = q->z * sl, o2 = 0;"),
    # memset and kernel arguments
    "ms_carry_ignores_pitch": ("a->shadow[dptr + y * pitch + i - a->base] = 0x00;",
                               "a->shadow[dptr + y * width + i - a->base] = 0x00;"),
    "ms_extent_whole_pitch": ("const uint64_t ext = (height - 1) * pitch + width;",
                              "const uint64_t ext = height * pitch;"),
    "ms_pitch_check_dropped": ("if (height > 1 && pitch < width) return OR_E_ARG;", ""),
    "ka_counts_full_masks_only": ("if (dev_v(ra, ptr[i] + k - ra->base) == 0) continue;",
                                  "if (dev_v(ra, ptr[i] + k - ra->base) != 0xFF) continue;"),
    "ka_write_short_by_one": ("memset(a->shadow + (ptr[i] - a->base), 0x00, bytes[i]);",
                              "memset(a->shadow + (ptr[i] - a->base), 0x00, bytes[i] - 1);"),
    "ka_write_as_src_flags": (
        "(void)device_side(s, ptr[i], bytes[i], &r->found_dst, &r->alloc_base_dst,\n"
        "                        &r->alloc_size_dst, &r->flags, OR_F_UNALLOC_DST, OR_F_OVERRUN_DST);",
        "(void)device_side(s, ptr[i], bytes[i], &r->found_dst, &r->alloc_base_dst,\n"
        "                        &r->alloc_size_dst, &r->flags, OR_F_UNALLOC_SRC, OR_F_OVERRUN_SRC);"),
    "ka_invalid_write_defines": ("if (reps[i].flags & (OR_F_UNALLOC_DST | OR_F_OVERRUN_DST)) continue;",
                                 "if (reps[i].flags & OR_F_UNALLOC_DST) continue;"),
    "ka_access_unchecked": ("if (access[i] == 0 || (access[i] & ~(OR_ARG_READ | OR_ARG_WRITE))) return OR_E_ARG;",
                            "if (access[i] == 0) return OR_E_ARG;"),
    # client requests (mark defined / undefined)
    "mark_range_from_base": ("if (!a || n > a->base + a->size - dptr) return OR_E_RANGE;\n  int st = materialise(a);",
                             "if (!a || n > a->size) return OR_E_RANGE;\n  int st = materialise(a);"),
    "mark_range_off_by_one": ("if (!a || n > a->base + a->size - dptr) return OR_E_RANGE;\n  int st = materialise(a);",
                              "if (!a || n >= a->base + a->size - dptr) return OR_E_RANGE;\n  int st = materialise(a);"),
    "mark_written_at_base": ("memset(a->shadow + (dptr - a->base), value, n);",
                             "memset(a->shadow, value, n);"),
    "mark_ignores_value": ("memset(a->shadow + (dptr - a->base), value, n);",
                           "memset(a->shadow + (dptr - a->base), 0x00, n);"),
    "mark_unallocated_accepted": ("if (!a || n > a->base + a->size - dptr) return OR_E_RANGE;\n  int st = materialise(a);",
                                  "if (!a) return OR_OK;\n  if (n > a->base + a->size - dptr) return OR_E_RANGE;\n  int st = materialise(a);"),
    "batch_not_validated_first": (
        "    int st = validate(s, kind[i], dst[i], src[i], n[i]);\n    if (st) {",
        "    int st = 0;\n    if (st) {"),
}


def _run_mutant(name: str) -> tuple[str, int, str]:
    old, new = MUTANTS[name]
    assert SRC.count(old) == 1, f"mutation {name}: anchor text not found exactly once"
    path = O.build_variant(SRC.replace(old, new), name)
    p = subprocess.run([sys.executable, os.path.join(HERE, "pins.py"), path],
                       capture_output=True, text=True, timeout=600)
    return name, p.returncode, (p.stdout + p.stderr)[-300:]


@pytest.mark.timeout(900)
def test_every_planted_mistake_is_caught():
    with ThreadPoolExecutor(max_workers=max(2, (os.cpu_count() or 2))) as ex:
        results = list(ex.map(_run_mutant, sorted(MUTANTS)))
    survivors = [(n, out) for n, rc, out in results if rc == 0]
    assert not survivors, f"pins missed these planted mistakes: {survivors}"


def test_real_oracle_passes_pins():
    p = subprocess.run([sys.executable, os.path.join(HERE, "pins.py")],
                       capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stdout + p.stderr

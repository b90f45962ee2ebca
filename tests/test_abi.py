"""libcg loads and exports every entry point include/cg.h declares; struct
layouts agree; host-only entry points work without a GPU.  No GPU needed."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import cg_synth as S
import oracle as O
import paper_1310_0901_gb300 as cg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = open(os.path.join(ROOT, "include", "cg.h")).read()


def declared_functions():
    body = re.sub(r"/\*.*?\*/", "", HEADER, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:cg_status|const char \*)\s*(cg_\w+)\s*\(", body,
                                 flags=re.M)))


def test_header_declares_the_entry_points():
    names = declared_functions()
    for must in ("cg_register_alloc", "cg_free", "cg_check_copy", "cg_check_batch",
                 "cg_create", "cg_destroy", "cg_bind_host_shadow"):
        assert must in names


def test_library_exports_every_declared_symbol():
    out = subprocess.run(["nm", "-D", "--defined-only", cg.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(cg_\w+)$", out, flags=re.M))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    bound = {n for n, _, _ in cg.SIGNATURES}
    assert set(declared_functions()) == bound


def test_struct_sizes_match_header_comments():
    assert ctypes.sizeof(cg.cg_copy) == 32
    assert ctypes.sizeof(cg.cg_report) == 120
    assert ctypes.sizeof(cg.cg_err_record) == 48
    assert ctypes.sizeof(cg.cg_karg) == 24 == cg.KARG_DTYPE.itemsize
    assert ctypes.sizeof(cg.cg_side3d) == 56 == ctypes.sizeof(O.OrSide3d)
    assert ctypes.sizeof(cg.cg_copy3d) == 144 == ctypes.sizeof(O.OrCopy3d)
    assert S.REQ_DTYPE.itemsize == 32


def test_flag_and_field_vocabulary_agrees_with_oracle():
    # both sides define the encoding independently; they must agree by name
    assert cg.FLAG_NAMES == O.FLAG_NAMES
    assert cg.FLAGS == O.FLAGS
    assert cg.REPORT_FIELDS == O.REPORT_FIELDS
    assert cg.RECORD_FIELDS == O.RECORD_FIELDS
    assert (cg.HTOD, cg.DTOH, cg.DTOD) == (O.HTOD, O.DTOH, O.DTOD)
    for k, v in O.STATUS.items():
        assert cg.STATUS[k] == v


def test_host_only_entry_points():
    assert cg.cg_version().decode() == "0.1.0"
    c = cg.cg_config()
    assert cg.cg_config_default(ctypes.byref(c)) == 0
    assert c.carry == 1 and c.strict_device_undef == 0
    rep = {f: 0 for f in cg.REPORT_FIELDS}
    rep.update(flags=cg.FLAGS["OVERRUN_SRC"], expected=8000000, found_src=4000000)
    text = cg.format_report(rep, cg.DTOH)
    assert "8000000" in text and "4000000" in text and "device->host" in text


def _brute_levels(reqs, modes=None):
    """Pairwise definition: request i depends on every earlier request j
    whose write range meets i's read or write range, or whose read range
    meets i's write range (host and device spaces apart).  With modes, a
    request writes only if it carries (bit 0) and reads a device source only
    if that source is valid (bit 1)."""
    def rw(i, q):
        k, d, s, n = int(q["kind"]), int(q["dst"]), int(q["src"]), int(q["n"])
        carries = modes is None or bool(modes[i] & 1)
        rdev = modes is None or bool(modes[i] & 2)
        if n == 0:
            return [], []
        w = [("d", d, d + n)] if carries else []
        if k == S.HTOD:
            return [("h", s, s + n)], w
        if k == S.DTOH:
            return ([("d", s, s + n)] if rdev else []), ([("h", d, d + n)] if carries else [])
        return ([("d", s, s + n)] if rdev else []), w

    def meet(xs, ys):
        return any(a[0] == b[0] and a[1] < b[2] and b[1] < a[2] for a in xs for b in ys)

    sets = [rw(i, q) for i, q in enumerate(reqs)]
    lv = []
    for i, (ri, wi) in enumerate(sets):
        best = -1
        for j in range(i):
            rj, wj = sets[j]
            if meet(wj, ri) or meet(wj, wi) or meet(rj, wi):
                best = max(best, lv[j])
        lv.append(best + 1)
    return lv


@pytest.mark.parametrize("seed", range(6))
def test_planner_matches_pairwise_definition(seed):
    rng = np.random.default_rng(seed)
    n = 300
    reqs = np.zeros(n, S.REQ_DTYPE)
    reqs["kind"] = rng.integers(1, 4, n)
    reqs["n"] = rng.integers(0, 40, n)
    reqs["dst"] = rng.integers(0, 400, n)
    reqs["src"] = rng.integers(0, 400, n)
    lv, nl = cg.plan_levels(reqs, carry=True)
    want = _brute_levels(reqs)
    assert lv.tolist() == want
    assert nl == max(want) + 1
    lv0, nl0 = cg.plan_levels(reqs, carry=False)
    assert not lv0.any() and nl0 == 1
    modes = rng.integers(0, 4, n).astype(np.uint8)
    lvm, _ = cg.plan_levels(reqs, carry=True, modes=modes)
    assert lvm.tolist() == _brute_levels(reqs, modes)


def test_planner_on_small_workload_is_exact():
    w = S.small(0)
    lv, nl = cg.plan_levels(w.reqs, carry=True)
    assert lv.tolist() == _brute_levels(w.reqs)


def _unit_ranges(q, u, modes):
    """(reads, writes) of one planning unit as (space, lo, hi) triples; a
    piece's host bytes are those of its rows of the anchor grid (512 bytes
    a row from the 16-byte boundary at or below src)."""
    kind, d, s, n = int(q["kind"]), int(q["dst"]), int(q["src"]), int(q["n"])
    carry = bool(modes[int(u["req"])] & 1)
    rdev = bool(modes[int(u["req"])] & 2)
    if n == 0:
        return [], []
    if int(u["row_hi"]):
        ax = s & 15
        lo = max(0, 512 * int(u["row_lo"]) - ax)
        hi = min(n, 512 * int(u["row_hi"]) - ax)
        return [("h", s + lo, s + hi)], []
    r, w = [], []
    if kind == 1:
        r.append(("h", s, s + n))
        if carry:
            w.append(("d", d, d + n))
    elif kind == 2:
        if carry:
            w.append(("h", d, d + n))
        if rdev:
            r.append(("d", s, s + n))
    else:
        if rdev:
            r.append(("d", s, s + n))
        if carry:
            w.append(("d", d, d + n))
    return r, w


@pytest.mark.parametrize("seed", range(4))
def test_unit_planner_orders_every_conflict(seed):
    """cg_plan_units: host reads longer than 1.5 pieces are cut into pieces
    that tile their rows in order, other copies stay whole, and every pair
    of units that conflict (one writes what the other reads or writes; a
    piece by its own rows' host bytes) runs in increasing levels.  Pieces
    cut the levels of long reads crossing many small writes."""
    rng = np.random.default_rng(seed)
    n, host_n, piece_rows = 400, 1 << 20, 8
    reqs = np.zeros(n, S.REQ_DTYPE)
    reqs["kind"] = rng.choice([1, 2, 3], n, p=[0.5, 0.4, 0.1])
    small = rng.random(n) < 0.7
    reqs["n"] = np.where(small, rng.integers(1, 6000, n), rng.integers(1, 200_000, n))
    reqs["src"] = rng.integers(0, host_n - 200_000, n)
    reqs["dst"] = rng.integers(0, host_n - 200_000, n)
    modes = rng.integers(0, 4, n).astype(np.uint8)
    modes[(reqs["kind"] == 1) & ~small] &= 2  # long host reads carry nothing
    units = cg.plan_units(reqs, host_n, piece_rows, carry=True, modes=modes)
    # pieces tile their copy's rows
    whole, pieces = 0, 0
    k = 0
    for i, q in enumerate(reqs):
        rows = ((((int(q["src"]) & 15) + int(q["n"]) + 15) >> 4) + 31) >> 5
        if units[k]["req"] != i:
            raise AssertionError(f"unit {k} is not request {i}")
        if units[k]["row_hi"] == 0:
            whole += 1
            k += 1
            continue
        assert q["kind"] == 1 and not modes[i] & 1 and rows > piece_rows * 1.5
        r = 0
        while k < len(units) and units[k]["req"] == i:
            assert (units[k]["row_lo"], units[k]["row_hi"]) == (r, min(rows, r + piece_rows))
            r += piece_rows
            k += 1
            pieces += 1
        assert r >= rows
    assert k == len(units) and pieces > 100
    sets = [_unit_ranges(reqs[int(u["req"])], u, modes) for u in units]

    def meet(xs, ys):
        return any(a[0] == b[0] and a[1] < b[2] and b[1] < a[2] for a in xs for b in ys)

    lv = units["level"]
    for j in range(len(units)):
        rj, wj = sets[j]
        for i in range(j):
            ri, wi = sets[i]
            if meet(wi, rj) or meet(wi, wj) or meet(ri, wj):
                assert lv[i] < lv[j], (i, j)
    # where no 64 KiB block of the host image holds more than 8 ranges in
    # part, the levels are exactly the pairwise definition's
    if seed < 2:
        sparse = reqs.copy()
        sparse["src"] = rng.integers(0, (64 << 20) - 200_000, n)
        sparse["dst"] = rng.integers(0, (64 << 20) - 200_000, n)
        su = cg.plan_units(sparse, 64 << 20, 256, carry=True, modes=modes)
        ss = [_unit_ranges(sparse[int(u["req"])], u, modes) for u in su]
        want = []
        for j in range(len(su)):
            rj, wj = ss[j]
            best = -1
            for i in range(j):
                ri, wi = ss[i]
                if meet(wi, rj) or meet(wi, wj) or meet(ri, wj):
                    best = max(best, want[i])
            want.append(best + 1)
        assert su["level"].tolist() == want
        # exact levels: a piece meets a subset of what its whole copy meets,
        # so pieces never need more levels than whole copies
        whole_only = cg.plan_units(sparse, 64 << 20, 0, carry=True, modes=modes)
        assert len(whole_only) == n and su["level"].max() <= whole_only["level"].max()
    assert not cg.plan_units(reqs, host_n, piece_rows, carry=False, modes=modes)["level"].any()


def test_unit_planner_keeps_adjacent_writes_apart_in_one_level():
    """Device->host copies into adjacent host ranges (sharing 64 KiB blocks
    of the image, never bytes) do not conflict: one level."""
    n, size = 48, (16 << 20) - 64
    reqs = np.zeros(n, S.REQ_DTYPE)
    reqs["kind"] = S.DTOH
    reqs["n"] = size
    reqs["dst"] = np.arange(n) * (16 << 20) + 7
    reqs["src"] = (np.arange(n) + 1) * (1 << 30)
    modes = np.full(n, 3, np.uint8)
    u = cg.plan_units(reqs, 1 << 30, 64, carry=True, modes=modes)
    assert len(u) == n and not u["level"].any()


def test_binding_structs_match_the_compiled_header(tmp_path):
    """Every ctypes mirror of a header struct has the size and field offsets a
    C compiler gives the header's declaration."""
    mirrors = {n: getattr(cg, n) for n in ("cg_copy", "cg_report", "cg_err_record", "cg_config",
                                           "cg_stats", "cg_side3d", "cg_copy3d", "cg_karg",
                                           "cg_request", "cg_result", "cg_serve_config",
                                           "cg_serve_stats")}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "cg.h"', "int main(void) {"]
    for n, t in mirrors.items():
        lines.append(f'  printf("{n} %zu\\n", sizeof({n}));')
        for f, _ in t._fields_:
            lines.append(f'  printf("{n}.{f} %zu\\n", offsetof({n}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "sizes.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "sizes"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                    str(exe)], check=True)
    got = dict(ln.split() for ln in subprocess.run([str(exe)], capture_output=True, text=True,
                                                   check=True).stdout.splitlines())
    for n, t in mirrors.items():
        assert int(got[n]) == ctypes.sizeof(t), n
        for f, _ in t._fields_:
            assert int(got[f"{n}.{f}"]) == getattr(t, f).offset, f"{n}.{f}"

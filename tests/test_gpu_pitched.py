"""GPU parity of pitched 2-D / 3-D copies and device arrays against the CPU
oracle, bit-exact (every verdict is an integer).

Mixed workloads (linear allocations and arrays, every kind, narrow record
fields to 24 KiB rows, tight / ragged / 512-rounded pitches, overruns,
freed targets, overlapping device->device copies) are applied to a libcg
context and to the oracle in the same order; each report, each API status,
and the final host V image, every allocation's and every array's shadow
must be equal.  The full-size 256 MiB transfers the benchmark times are
compared with the oracle in full."""
from __future__ import annotations

import collections
import ctypes

import numpy as np
import pytest

import cg_synth as S
import oracle as O
from tests import gpu_util as U

pytestmark = pytest.mark.gpu

HTOD, DTOH, DTOD = S.HTOD, S.DTOH, S.DTOD


@pytest.fixture(scope="module")
def cg():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1310_0901_gb300 as m
    return m


def _pair(w, carry=True, **cfg):
    ctx, orc, (a, v) = U.make_pair(w.image, w.table, carry=carry, **cfg)
    for h, W, H, D in w.arrays:
        assert ctx.register_array(h, W, H, D) == 0
        assert orc.register_array(h, W, H, D) == 0
    return ctx, orc, v


def _same_state(ctx, orc, v, w):
    U.assert_same_state(ctx, orc, v, w.table)
    for h, W, H, D in w.arrays:
        g = ctx.read_array_shadow(h, 0, W * H * D)
        o = orc.read_array_v(h, 0, W * H * D)
        assert np.array_equal(g, o), f"array {h:#x} shadow differs at {np.nonzero(g != o)[0][:8]}"


def _both(ctx, orc, q):
    args = (q["kind"], q["dst"], q["src"], q["width"], q["height"], q["depth"])
    st_g, g = ctx.check_copy3d(*args)
    st_o, o = orc.check_copy3d(*args)
    return st_g, g, st_o, o


@pytest.mark.parametrize("seed,carry,engine", [(0, True, 0), (1, True, 0), (2, False, 0),
                                               (3, True, 1)])
def test_pitched_workload_matches_oracle(cg, seed, carry, engine):
    w = S.pitched(seed)
    ctx, orc, v = _pair(w, carry, scan_engine=engine)
    seen = collections.Counter()
    for i, q in enumerate(w.copies):
        st_g, g, st_o, o = _both(ctx, orc, q)
        assert st_g == st_o, (i, q, st_g, st_o, cg.cg_last_error())
        if st_o == 0:
            U.assert_same_report(g, o, f"copy {i} {q}")
            for name, bit in O.FLAGS.items():
                if o["flags"] & bit:
                    seen[name] += 1
            seen["narrow" if q["width"] <= 64 else "wide" if q["width"] > 2048 else "mid"] += 1
            seen["3d" if q["depth"] > 1 else "2d"] += 1
            seen["array"] += q["dst"]["is_array"] | q["src"]["is_array"]
        if i % 100 == 99:
            _same_state(ctx, orc, v, w)
    _same_state(ctx, orc, v, w)
    # the mix exercised every class it is meant to
    for k in ("HOST_UNDEF", "HOST_UNADDR", "OVERRUN_DST", "DEV_UNDEF_SRC", "narrow", "mid",
              "wide", "3d", "array"):
        assert seen[k] > 0, (k, seen)
    if seed == 0:
        assert seen["DTOD_OVERLAP"] > 0 and seen["UNALLOC_DST"] + seen["UNALLOC_SRC"] > 0, seen


def test_strided_records_footnote(cg):
    """A field of an array of records (the footnote's strided host access):
    the pitched check of the 16-byte field reports only what was planted in
    the field, a plain check of the same span also reports the padding."""
    rng = S.rng_for(5)
    rec, pay, nrec = 24, 16, 1 << 16
    n_img = rec * nrec
    v = np.zeros(n_img, np.uint8)
    v.reshape(nrec, rec)[:, pay:] = 0xFF                         # padding never written
    planted = rng.choice(nrec * pay, 300, replace=False)         # payload bytes made undefined
    rows, cols = planted // pay, planted % pay
    v.reshape(nrec, rec)[rows, cols] = rng.integers(1, 256, planted.size).astype(np.uint8)
    img = S.HostImage(S.pack_a(np.ones(n_img, bool)), v, [], None)
    base = 1 << 40
    table = S.AllocTable(np.array([base], np.uint64), np.array([4 << 20], np.uint64),
                         np.zeros(0, np.int64))
    w = S.PitchedWorkload(img, table, [], [])
    ctx, orc, vt = _pair(w)
    q = dict(kind=HTOD, dst=S.side3d(base, pay, 0), src=S.side3d(0, rec, 0), width=pay,
             height=nrec, depth=1)
    st_g, g, st_o, o = _both(ctx, orc, q)
    assert st_g == st_o == 0
    U.assert_same_report(g, o, "records")
    assert g["n_undef"] == 300 and g["n_unaddr"] == 0
    assert g["first_undef_off"] == int(np.sort(rows * pay + cols)[0])
    span = (nrec - 1) * rec + pay
    st, g1 = ctx.check_copy(HTOD, base + (2 << 20), 0, span)
    assert st == 0 and g1["n_undef"] == 300 + (nrec - 1) * (rec - pay)
    assert orc.check_copy(HTOD, base + (2 << 20), 0, span) == (0, g1)
    _same_state(ctx, orc, vt, w)


def test_pitched_edges(cg):
    """Statuses and reports of the corner cases equal the oracle's: empty
    copies (no range check), rows closer than the width, slices closer
    than the rows, a host extent past the image, geometry beyond 64 bits,
    an array as the host side, reserved fields, unknown and destroyed
    arrays, a single row with no pitch, exact fits and one byte over."""
    w = S.pitched(4, n_copies=1)
    ctx, orc, v = _pair(w)
    b0, s0 = int(w.table.base[0]), int(w.table.size[0])
    h0 = w.arrays[0]
    cases = [
        (HTOD, S.side3d(b0), S.side3d(0), 0, 9, 9),
        (HTOD, S.side3d(12345, array=True), S.side3d(1 << 50), 5, 5, 0),
        (HTOD, S.side3d(b0, 7), S.side3d(0, 8), 8, 2, 1),
        (DTOH, S.side3d(0, 8, 1), S.side3d(b0, 8, 2), 8, 2, 2),
        (HTOD, S.side3d(b0, 16), S.side3d(w.image.n - 100, 64), 16, 3, 1),
        (HTOD, S.side3d(b0, 1 << 62, 8), S.side3d(0, 8, 8), 8, 2, 2),
        (HTOD, S.side3d(b0), S.side3d(h0[0], array=True), 4, 1, 1),
        (HTOD, S.side3d(0x7777, array=True), S.side3d(0, 4), 4, 1, 1),
        (HTOD, S.side3d(b0, 0, 0, 3), S.side3d(10, 0), 100, 1, 1),
        (HTOD, S.side3d(b0 + s0 - (3 * 100 + 10), 100), S.side3d(0, 10), 10, 4, 1),
        (HTOD, S.side3d(b0 + s0 - (3 * 100 + 9), 100), S.side3d(0, 10), 10, 4, 1),
        (HTOD, S.side3d(h0[0], 0, 0, h0[1] - 4, h0[2] - 1, h0[3] - 1, array=True),
         S.side3d(0, 4), 4, 1, 1),
        (HTOD, S.side3d(h0[0], 0, 0, h0[1] - 4, h0[2] - 1, h0[3] - 1, array=True),
         S.side3d(0, 5), 5, 1, 1),
        (DTOD, S.side3d(h0[0], 0, 0, 1, 0, 0, array=True),
         S.side3d(h0[0], 0, 0, 0, 0, 0, array=True), min(64, h0[1] - 1), 1, 1),
        (DTOD, S.side3d(b0 + 8, 64), S.side3d(b0, 64), 40, 20, 1),
    ]
    for i, (kind, d, s, ww, hh, dd) in enumerate(cases):
        q = dict(kind=kind, dst=d, src=s, width=ww, height=hh, depth=dd)
        st_g, g, st_o, o = _both(ctx, orc, q)
        assert st_g == st_o, (i, st_g, st_o, cg.cg_last_error())
        if st_o == 0:
            U.assert_same_report(g, o, f"edge case {i}")
    # reserved fields
    q = cg.copy3d(HTOD, S.side3d(b0), S.side3d(0), 4, 1, 1)
    q.src.reserved = 1
    r = cg.cg_report()
    assert cg.cg_check_copy3d(ctx.handle, ctypes.byref(q), ctypes.byref(r), None) == -1
    # arrays: destroy, double, unknown; a destroyed array is unallocated
    h = w.arrays[1][0]
    assert ctx.free_array(h) == orc.free_array(h) == "OK"
    assert ctx.free_array(h) == orc.free_array(h) == "DOUBLE"
    assert ctx.free_array(0x1234) == orc.free_array(0x1234) == "UNKNOWN"
    q = dict(kind=HTOD, dst=S.side3d(h, array=True), src=S.side3d(0, 4), width=4, height=1,
             depth=1)
    st_g, g, st_o, o = _both(ctx, orc, q)
    assert st_g == st_o == 0 and g["flags"] & O.FLAGS["UNALLOC_DST"]
    U.assert_same_report(g, o, "destroyed array")
    assert ctx.register_array(h, 64, 2, 1) == orc.register_array(h, 64, 2, 1) == 0
    assert ctx.register_array(h, 64, 2, 1) == orc.register_array(h, 64, 2, 1) == -6
    w.arrays[1] = (h, 64, 2, 1)
    _same_state(ctx, orc, v, w)


def test_pitched_async_equals_sync(cg):
    """cg_check_copy3d_async writes the same report into device memory, and
    a copy with nothing to read still gets its report."""
    import torch
    w = S.pitched(5, n_copies=40)
    c1, orc, v1 = _pair(w)
    c2, _, v2 = _pair(w)
    reps = torch.zeros((len(w.copies) + 1, cg.REPORT_DTYPE.itemsize), dtype=torch.uint8,
                       device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    want = []
    for i, q in enumerate(w.copies):
        st, r = c1.check_copy3d(q["kind"], q["dst"], q["src"], q["width"], q["height"], q["depth"])
        want.append((st, r))
        qq = cg.copy3d(q["kind"], q["dst"], q["src"], q["width"], q["height"], q["depth"])
        st2 = cg.cg_check_copy3d_async(c2.handle, ctypes.byref(qq), reps[i].data_ptr(), stream)
        assert st2 == st
    # device->device from a freed allocation to a live one: nothing to read
    fb = int(w.table.base[w.table.freed[0]])
    lb = int(w.table.base[np.setdiff1d(np.arange(len(w.table.base)), w.table.freed)[0]])
    qq = cg.copy3d(DTOD, S.side3d(lb, 8), S.side3d(fb, 8), 8, 2, 1)
    assert cg.cg_check_copy3d_async(c2.handle, ctypes.byref(qq), reps[-1].data_ptr(), stream) == 0
    torch.cuda.synchronize()
    got = np.frombuffer(reps.cpu().numpy().tobytes(), dtype=cg.REPORT_DTYPE)
    for i, (st, r) in enumerate(want):
        if st == 0:
            assert {k: int(got[i][k]) for k in got.dtype.names} == r, i
    st_o, o = orc.check_copy3d(DTOD, S.side3d(lb, 8), S.side3d(fb, 8), 8, 2)
    assert {k: int(got[-1][k]) for k in got.dtype.names} == o
    assert np.array_equal(v1.cpu().numpy(), v2.cpu().numpy())


@pytest.mark.parametrize("which", sorted(S.PITCHED_LARGE))
def test_pitched_large_matches_oracle(cg, which):
    """The benchmark's full-size transfers (256 MiB of payload), in its
    launch configuration, against the oracle in full: report and the whole
    carried device shadow; and the planted payload truth."""
    import torch
    w = S.pitched_large(which)
    q = w.copies[0]
    ctx, orc, (a, v) = U.make_pair(w.image, w.table)
    rep = torch.zeros(cg.REPORT_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    qq = cg.copy3d(q["kind"], q["dst"], q["src"], q["width"], q["height"], q["depth"])
    st = cg.cg_check_copy3d_async(ctx.handle, ctypes.byref(qq), rep.data_ptr(),
                                  torch.cuda.current_stream().cuda_stream)
    assert st == 0, cg.cg_last_error()
    torch.cuda.synchronize()
    r = np.frombuffer(rep.cpu().numpy().tobytes(), dtype=cg.REPORT_DTYPE)[0]
    got = {k: int(r[k]) for k in r.dtype.names}
    wd, hh, hp = q["width"], q["height"], q["src"]["pitch"]
    payload = np.lib.stride_tricks.as_strided(w.image.v, shape=(hh, wd), strides=(hp, 1))
    assert got["n_undef"] == int((payload != 0).sum())      # planted runs in the payload only
    st_o, o = orc.check_copy3d(q["kind"], q["dst"], q["src"], wd, hh, 1)
    assert st_o == 0
    U.assert_same_report(got, o, which)
    b, s = int(w.table.base[0]), int(w.table.size[0])
    assert np.array_equal(ctx.read_device_shadow(b, s), orc.read_dev_v(b, s))


def test_pitched_host_resident_image(cg):
    """An image in pinned host memory (read in place, register kernels for
    every row length): the mixed workload still equals the oracle."""
    import torch
    w = S.pitched(6, n_copies=150)
    n = w.image.n
    a_h = torch.from_numpy(w.image.a_bits[: n // 8].copy()).pin_memory()
    v_h = torch.from_numpy(w.image.v.copy()).pin_memory()
    ctx = cg.Context()
    ctx.bind_host_shadow(a_h, v_h)
    orc = O.Oracle(w.image.a_bits, w.image.v)
    bases, sizes = U.sorted_table(w.table)
    assert not ctx.register_allocs(bases, sizes).any()
    for b, s_ in zip(bases, sizes):
        assert orc.register_alloc(int(b), int(s_)) == 0
    for j in w.table.freed:
        assert ctx.free(int(w.table.base[j])) == orc.free(int(w.table.base[j])) == "OK"
    for h, W, H, D in w.arrays:
        assert ctx.register_array(h, W, H, D) == orc.register_array(h, W, H, D) == 0
    wide = 0
    for i, q in enumerate(w.copies):
        st_g, g, st_o, o = _both(ctx, orc, q)
        assert st_g == st_o, (i, st_g, st_o)
        if st_o == 0:
            U.assert_same_report(g, o, f"host image copy {i}")
            wide += q["width"] >= 4096
    assert wide > 0
    torch.cuda.synchronize()
    assert np.array_equal(v_h.numpy(), orc.read_host_v())

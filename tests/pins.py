"""Pins for the CPU oracle: facts fixed by the paper or by mathematics that a
plausible mistake in the oracle would break.

Each ``pin_*`` takes a loaded oracle library and raises ``AssertionError`` if
the oracle disagrees.  ``tests/test_oracle_pins.py`` runs them against the
real oracle; ``tests/test_oracle_mutants.py`` plants mistakes in a copy of the
oracle source and checks that some pin fails for every mistake.

Where a pin needs an expected value it comes from (a) the paper (the
Listing 5 fixture), (b) construction (the inputs are built from a list of
intended byte classes or planted runs), (c) a different formulation (set
membership over every address instead of a sorted-table search; Python's
slice assignment for memmove), or (d) an invariant.
"""
from __future__ import annotations

import itertools
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import cg_synth as S  # noqa: E402
import oracle as O  # noqa: E402

HTOD, DTOH, DTOD = O.HTOD, O.DTOH, O.DTOD
F = O.FLAGS

# (A bit, V byte) states a host byte can take; the class each one belongs to
# is written down here as data: unaddressable wins, else any set V bit means
# undefined (Sec. 1.1 bit precision; readings R1-R3).
BYTE_STATES = [
    (0, 0x00, O.BYTE_UNADDR), (0, 0x01, O.BYTE_UNADDR), (0, 0x80, O.BYTE_UNADDR),
    (0, 0xFF, O.BYTE_UNADDR), (1, 0x00, O.BYTE_GOOD), (1, 0x01, O.BYTE_UNDEF),
    (1, 0x80, O.BYTE_UNDEF), (1, 0xFF, O.BYTE_UNDEF),
]


def _image(addressable: np.ndarray, v: np.ndarray):
    return S.pack_a(addressable.astype(bool)), np.ascontiguousarray(v, dtype=np.uint8)


def _expect_from_classes(classes):
    n_unaddr = sum(1 for c in classes if c == O.BYTE_UNADDR)
    n_undef = sum(1 for c in classes if c == O.BYTE_UNDEF)
    bad = [i for i, c in enumerate(classes) if c != O.BYTE_GOOD]
    fu = [i for i, c in enumerate(classes) if c == O.BYTE_UNADDR]
    fd = [i for i, c in enumerate(classes) if c == O.BYTE_UNDEF]
    return dict(
        n_good=len(classes) - n_unaddr - n_undef, n_unaddr=n_unaddr, n_undef=n_undef,
        first_bad_off=bad[0] if bad else -1,
        first_bad_kind=classes[bad[0]] if bad else 0,
        first_unaddr_off=fu[0] if fu else -1, first_undef_off=fd[0] if fd else -1)


def _sub(d: dict, keys) -> dict:
    return {k: d[k] for k in keys}


SCAN_KEYS = ["n_good", "n_unaddr", "n_undef", "first_bad_off", "first_bad_kind",
             "first_unaddr_off", "first_undef_off"]


# --------------------------------------------------------------------- pins

def pin_listing5(lib):
    """Sec. 4, Listings 2 and 5: a device->host copy of size*sizeof(double)
    from an allocation of size*sizeof(float) is reported as too large, with
    8000000 bytes expected and 4000000 found."""
    g = json.load(open(os.path.join(HERE, "golden", "listing5_dtoh_overrun.json")))
    n = g["copy_bytes"]
    a_bits, v = _image(np.ones(n, bool), np.full(n, 0xFF, np.uint8))
    o = O.Oracle(a_bits, v, lib=lib)
    c, a, b = 0x7f0000000000, 0x7f0000400000, 0x7f0000c00000
    assert o.register_alloc(c, g["alloc_c_bytes"]) == 0
    assert o.register_alloc(a, g["alloc_a_bytes"]) == 0
    assert o.register_alloc(b, g["alloc_b_bytes"]) == 0
    st, r = o.check_copy(DTOH, 0, c, n)
    assert st == 0
    assert r["flags"] & F["OVERRUN_SRC"], r
    assert not r["flags"] & (F["UNALLOC_SRC"] | F["UNALLOC_DST"] | F["OVERRUN_DST"])
    assert r["expected"] == g["expected"]
    assert r["found_src"] == g["found"]
    assert r["alloc_base_src"] == c and r["alloc_size_src"] == g["alloc_c_bytes"]
    # the correctly sized copy of c is in range
    st, r = o.check_copy(DTOH, 0, c, g["alloc_c_bytes"])
    assert st == 0 and not r["flags"] & (F["OVERRUN_SRC"] | F["UNALLOC_SRC"])
    assert r["found_src"] == g["alloc_c_bytes"]
    # the two inputs (doubles) copy in range
    for p in (a, b):
        st, r = o.check_copy(HTOD, p, 0, n)
        assert st == 0 and not r["flags"] & (F["OVERRUN_DST"] | F["UNALLOC_DST"]), r


def pin_htod_bytes_by_construction(lib, max_n: int = 4):
    """Every assignment of the 8 (A, V) states to n <= 4 bytes, at every A-bit
    phase 0..15: counts and first offsets must equal those of the class list
    the input was built from.  The surrounding bytes hold other states, so a
    read outside the copy changes the answer."""
    img_n = 64
    noise_rng = np.random.default_rng(7)
    for n in range(1, max_n + 1):
        combos = list(itertools.product(range(len(BYTE_STATES)), repeat=n))
        if n == 4:  # thin the 4096 patterns out but keep every state per slot
            combos = combos[::3]
        for ci, combo in enumerate(combos):
            h = ci % 16 + 8
            addr = noise_rng.integers(0, 2, img_n).astype(bool)
            v = noise_rng.integers(0, 256, img_n).astype(np.uint8)
            for i, st in enumerate(combo):
                addr[h + i] = bool(BYTE_STATES[st][0])
                v[h + i] = BYTE_STATES[st][1]
            classes = [BYTE_STATES[st][2] for st in combo]
            a_bits, vv = _image(addr, v)
            o = O.Oracle(a_bits, vv, lib=lib)
            assert o.register_alloc(1 << 20, 4096) == 0
            stat, r = o.check_copy(HTOD, (1 << 20) + 16, h, n)
            assert stat == 0
            exp = _expect_from_classes(classes)
            assert _sub(r, SCAN_KEYS) == exp, (combo, h, r, exp)
            want_flags = (F["HOST_UNADDR"] if exp["n_unaddr"] else 0) | \
                         (F["HOST_UNDEF"] if exp["n_undef"] else 0)
            assert r["flags"] == want_flags, (combo, r["flags"])
            o.close()


def pin_dtoh_bytes_by_construction(lib):
    """Device->host: the destination's A bit and the device source's V byte
    (placed there by an exact host->device carry from a fully addressable
    staging area) decide each byte's class."""
    rng = np.random.default_rng(11)
    for trial in range(400):
        n = int(rng.integers(1, 9))
        states = rng.integers(0, len(BYTE_STATES), n)
        img_n = 128
        addr = rng.integers(0, 2, img_n).astype(bool)
        v = rng.integers(0, 256, img_n).astype(np.uint8)
        stage = 96  # staging area: addressable, V = the device values wanted
        addr[stage:stage + n] = True
        h = int(rng.integers(0, 40))
        for i, st in enumerate(states):
            addr[h + i] = bool(BYTE_STATES[st][0])
            v[stage + i] = BYTE_STATES[st][1]
        classes = [BYTE_STATES[st][2] for st in states]
        a_bits, vv = _image(addr, v)
        o = O.Oracle(a_bits, vv, lib=lib)
        dev = 0x5000_0000
        assert o.register_alloc(dev, 256) == 0
        st0, _ = o.check_copy(HTOD, dev + 7, stage, n)
        assert st0 == 0
        stat, r = o.check_copy(DTOH, h, dev + 7, n)
        assert stat == 0
        exp = _expect_from_classes(classes)
        assert _sub(r, SCAN_KEYS) == exp, (trial, r, exp)
        want = (F["HOST_UNADDR"] if exp["n_unaddr"] else 0) | \
               (F["DEV_UNDEF_SRC"] if exp["n_undef"] else 0)
        assert r["flags"] == want
        o.close()


def _owner(layout, addr):
    for k, (b, s) in enumerate(layout):
        if b <= addr < b + s:
            return k
    return None


def _range_truth(layout, d, n):
    """Set membership over every address: the copy is in range iff every
    address of [d, d+n) belongs to one and the same allocation."""
    own = _owner(layout, d)
    if own is None:
        return "UNALLOC", 0
    found = 0
    a = d
    while _owner(layout, a) == own:
        found += 1
        a += 1
    ok = all(_owner(layout, x) == own for x in range(d, d + n))
    return ("OK" if ok else "OVERRUN"), found


def pin_range_bruteforce(lib, trials: int = 300):
    """Up to three allocations in a 64-address space, random copies: the
    verdict and the found count equal the set-membership truth (Sec. 2
    itemize; R7, R8)."""
    rng = np.random.default_rng(3)
    v = np.zeros(128, np.uint8)
    a_bits, vv = _image(np.ones(128, bool), v)
    for t in range(trials):
        k = int(rng.integers(0, 4))
        cuts = np.sort(rng.choice(np.arange(0, 65), size=2 * k, replace=False))
        layout = [(int(cuts[2 * i]), int(cuts[2 * i + 1] - cuts[2 * i])) for i in range(k)]
        layout = [(b, s) for b, s in layout if s > 0]
        o = O.Oracle(a_bits, vv, lib=lib)
        base0 = 1 << 32
        for b, s in layout:
            assert o.register_alloc(base0 + b, s) == 0
        for _ in range(30):
            d = int(rng.integers(0, 64))
            n = int(rng.integers(1, 40))
            verdict, found = _range_truth(layout, d, n)
            stat, r = o.check_copy(HTOD, base0 + d, 0, n)
            assert stat == 0
            got = "UNALLOC" if r["flags"] & F["UNALLOC_DST"] else \
                "OVERRUN" if r["flags"] & F["OVERRUN_DST"] else "OK"
            assert got == verdict, (layout, d, n, r)
            assert r["found_dst"] == found, (layout, d, n, r["found_dst"], found)
            if verdict != "UNALLOC":
                b, s = layout[_owner(layout, d)]
                assert (r["alloc_base_dst"], r["alloc_size_dst"]) == (base0 + b, s)
        o.close()


def pin_free_sequences(lib):
    """Frees of live, interior, already freed and unknown pointers; refused
    registrations (the error classes named for frees; R13, R14)."""
    o = O.Oracle(*_image(np.ones(16, bool), np.zeros(16, np.uint8)), lib=lib)
    assert o.register_alloc(100, 10) == 0
    assert o.register_alloc(105, 10) == -6          # overlaps [100, 110)
    assert o.register_alloc(90, 11) == -6           # ends inside
    assert o.register_alloc(90, 10) == 0            # touches, no overlap
    assert o.register_alloc(200, 0) == -4           # zero size
    assert o.register_alloc((1 << 64) - 8, 16) == -5  # wraps
    assert o.free(105) == "INTERIOR"
    assert o.free(100) == "OK"
    assert o.free(100) == "DOUBLE"
    assert o.free(300) == "UNKNOWN"
    assert o.free(90) == "OK"
    assert o.free(90) == "DOUBLE"
    assert o.live_count() == 0
    o.close()


def pin_free_sequences_reuse(lib):
    """A freed base that a later allocation covers is no longer a double
    free target; after that allocation's free it is unknown, not double."""
    o = O.Oracle(*_image(np.ones(16, bool), np.zeros(16, np.uint8)), lib=lib)
    assert o.register_alloc(100, 10) == 0
    assert o.free(100) == "OK"
    assert o.register_alloc(96, 20) == 0
    assert o.free(100) == "INTERIOR"
    assert o.free(96) == "OK"
    assert o.free(100) == "UNKNOWN"
    assert o.free(96) == "DOUBLE"
    assert o.register_alloc(96, 4) == 0
    assert o.free(96) == "OK"
    assert o.live_count() == 0
    o.close()


def pin_generator_truth(lib):
    """Counts of a host->device scan equal what the generator planted: the
    undefined bytes are the union of the planted runs (all masks nonzero by
    construction) minus the planted unaddressable positions."""
    rng = S.rng_for(5)
    img = S.host_image_runs(rng, 1 << 16, 0.02, 8.0, 0.5, 0.003)
    undef = np.zeros(img.n, bool)
    for s0, ln in img.undef_runs:
        undef[s0:s0 + ln] = True
    unaddr = np.zeros(img.n, bool)
    unaddr[img.unaddr] = True
    o = O.Oracle(img.a_bits, img.v, carry=False, lib=lib)
    assert o.register_alloc(1 << 40, 1 << 16) == 0
    for _ in range(300):
        n = int(rng.integers(1, 5000))
        h = int(rng.integers(0, img.n - n + 1))
        st, r = o.check_copy(HTOD, 1 << 40, h, n)
        assert st == 0
        ua = unaddr[h:h + n]
        ud = undef[h:h + n] & ~ua
        assert r["n_unaddr"] == int(ua.sum())
        assert r["n_undef"] == int(ud.sum())
        assert r["first_unaddr_off"] == (int(np.argmax(ua)) if ua.any() else -1)
        assert r["first_undef_off"] == (int(np.argmax(ud)) if ud.any() else -1)
    o.close()


def pin_invariants(lib):
    """good + unaddr + undef = n; the first bad offset is the smaller of the
    per-class first offsets; counts add up when a copy is split in two."""
    rng = S.rng_for(9)
    img = S.host_image_runs(rng, 1 << 15, 0.05, 8.0, 0.5, 0.01)
    o = O.Oracle(img.a_bits, img.v, carry=False, lib=lib)
    assert o.register_alloc(1 << 30, 1 << 15) == 0
    for _ in range(300):
        n = int(rng.integers(2, 3000))
        h = int(rng.integers(0, img.n - n + 1))
        k = int(rng.integers(1, n))
        _, w = o.check_copy(HTOD, 1 << 30, h, n)
        _, a = o.check_copy(HTOD, 1 << 30, h, k)
        _, b = o.check_copy(HTOD, (1 << 30) + k, h + k, n - k)
        assert w["n_good"] + w["n_unaddr"] + w["n_undef"] == n
        for key in ("n_good", "n_unaddr", "n_undef"):
            assert w[key] == a[key] + b[key]
        for key in ("first_unaddr_off", "first_undef_off", "first_bad_off"):
            want = a[key] if a[key] >= 0 else (b[key] + k if b[key] >= 0 else -1)
            assert w[key] == want
        firsts = [x for x in (w["first_unaddr_off"], w["first_undef_off"]) if x >= 0]
        assert w["first_bad_off"] == (min(firsts) if firsts else -1)
    o.close()


def pin_carry_roundtrip(lib):
    """Sec. 5 (definedness follows the data): host->device then device->host
    of fully addressable bytes restores the V masks exactly; a fresh
    allocation reads back as undefined (R6); a failed copy carries nothing
    (R11); unaddressable destination bytes keep their masks."""
    rng = S.rng_for(13)
    n_img = 1 << 14
    v = rng.integers(0, 256, n_img).astype(np.uint8)
    v[rng.random(n_img) < 0.5] = 0
    addr = np.ones(n_img, bool)
    addr[8192:] = rng.random(n_img - 8192) > 0.2   # second half: holes
    a_bits, vv = _image(addr, v)
    o = O.Oracle(a_bits, vv, lib=lib)
    dev = 1 << 36
    assert o.register_alloc(dev, 4096) == 0
    # fresh allocation -> every addressable destination byte becomes 0xFF
    st, r = o.check_copy(DTOH, 8192, dev, 1000)
    assert st == 0
    hv = o.read_host_v(8192, 1000)
    exp = np.where(addr[8192:9192], 0xFF, v[8192:9192]).astype(np.uint8)
    assert np.array_equal(hv, exp)
    assert r["n_undef"] == int(addr[8192:9192].sum())
    assert r["n_unaddr"] == int((~addr[8192:9192]).sum())
    # round trip over the fully addressable first half
    st, _ = o.check_copy(HTOD, dev + 100, 0, 3000)
    assert st == 0
    assert np.array_equal(o.read_dev_v(dev + 100, 3000), v[:3000])
    st, _ = o.check_copy(DTOH, 4000, dev + 100, 3000)
    assert np.array_equal(o.read_host_v(4000, 3000), v[:3000])
    # the untouched device bytes are still undefined
    assert np.all(o.read_dev_v(dev, 100) == 0xFF)
    # unaddressable source bytes arrive on the device undefined
    st, r = o.check_copy(HTOD, dev + 3200, 9500, 800)
    assert st == 0 and r["n_unaddr"] == int((~addr[9500:10300]).sum())
    got = o.read_dev_v(dev + 3200, 800)
    holes = ~addr[9500:10300]
    assert np.all(got[holes] == 0xFF)
    assert np.array_equal(got[~holes], v[9500:10300][~holes])
    # an overrunning copy carries nothing
    before = o.read_dev_v(dev, 4096).copy()
    st, r = o.check_copy(HTOD, dev + 4000, 8192, 200)
    assert r["flags"] & F["OVERRUN_DST"]
    assert np.array_equal(o.read_dev_v(dev, 4096), before)
    # n == 0 is a no-op (R9) even on a wild pointer
    st, r = o.check_copy(HTOD, 12345, 0, 0)
    assert st == 0 and r["flags"] == 0 and r["first_bad_off"] == -1
    o.close()


def pin_mark(lib):
    """The Memcheck-style client requests (mark a device range defined or
    undefined; the outlook's way for callers to declare kernel output, R6):
    a mark rewrites exactly [dptr, dptr + n) of the allocation holding dptr,
    with 0x00 (defined) or 0xFF (undefined), and a device->host copy of the
    allocation then counts what the marks left, by construction.  A mark
    that is not wholly inside one live allocation (no allocation, a freed
    one, or running past the end of the one holding dptr) is refused with
    E_RANGE and changes nothing; n = 0 is a no-op."""
    n_img = 1 << 13
    v = np.zeros(n_img, np.uint8)
    a_bits, vv = _image(np.ones(n_img, bool), v)
    o = O.Oracle(a_bits, vv, lib=lib)
    dev, size = 1 << 40, 4096
    assert o.register_alloc(dev, size) == 0
    assert o.register_alloc(dev + size, 512) == 0        # adjacent, never combined
    assert o.register_alloc(1 << 41, 256) == 0
    assert o.free(1 << 41) == "OK"
    model = np.full(size, 0xFF, np.uint8)                # fresh: all undefined (R6)
    rng = S.rng_for(29)
    for step in range(60):
        n = int(rng.integers(1, 700))
        off = int(rng.integers(0, size - n + 1))
        val = 0x00 if step % 3 else 0xFF
        assert o.mark(dev + off, n, val) == 0
        model[off:off + n] = val
        assert np.array_equal(o.read_dev_v(dev, size), model), step
    # a device->host copy of the whole allocation into fully addressable
    # host bytes: the undefined count and first offset follow from the model
    st, r = o.check_copy(DTOH, 0, dev, size)
    assert st == 0
    bad = np.nonzero(model)[0]
    assert r["n_undef"] == bad.size and r["n_good"] == size - bad.size
    assert r["first_undef_off"] == (int(bad[0]) if bad.size else -1)
    assert np.array_equal(o.read_host_v(0, size), model)
    # refusals: nothing changes
    before = o.read_dev_v(dev, size).copy()
    nxt = o.read_dev_v(dev + size, 512).copy()
    assert o.mark(dev + 100, size - 99, 0x00) == -8      # one byte past the end
    assert o.mark(dev + size - 1, 2, 0x00) == -8         # runs into the neighbour
    assert o.mark(dev - 1, 2, 0x00) == -8                # starts before any allocation
    assert o.mark(1 << 41, 16, 0x00) == -8               # freed
    assert o.mark(1 << 30, 16, 0x00) == -8               # never allocated
    assert np.array_equal(o.read_dev_v(dev, size), before)
    assert np.array_equal(o.read_dev_v(dev + size, 512), nxt)
    # the largest accepted marks end exactly at the end
    assert o.mark(dev + 100, size - 100, 0x00) == 0
    assert o.mark(dev + size + 7, 505, 0xFF) == 0
    model[100:] = 0x00
    assert np.array_equal(o.read_dev_v(dev, size), model)
    assert o.mark(12345, 0, 0x00) == 0                   # n = 0: a no-op
    o.close()


def pin_dtod_memmove(lib):
    """Device->device carries like memmove, compared against Python's slice
    assignment (which reads the whole source before writing); overlapping
    copies raise the overlap warning (R12).  A chain X->Y->Z leaves Z as
    a direct X->Z copy would."""
    rng = S.rng_for(17)
    n_img = 4096
    v = rng.integers(0, 256, n_img).astype(np.uint8)
    a_bits, vv = _image(np.ones(n_img, bool), v)
    o = O.Oracle(a_bits, vv, lib=lib)
    dev = 1 << 33
    assert o.register_alloc(dev, 4096) == 0
    assert o.check_copy(HTOD, dev, 0, 4096)[0] == 0
    model = bytearray(v.tobytes())
    for _ in range(200):
        n = int(rng.integers(1, 600))
        s0 = int(rng.integers(0, 4096 - n + 1))
        d0 = int(np.clip(s0 + rng.integers(-n, n + 1), 0, 4096 - n))
        st, r = o.check_copy(DTOD, dev + d0, dev + s0, n)
        assert st == 0
        model[d0:d0 + n] = model[s0:s0 + n]
        assert bool(r["flags"] & F["DTOD_OVERLAP"]) == (abs(d0 - s0) < n)
        assert o.read_dev_v(dev, 4096).tobytes() == bytes(model)
    # chain X -> Y -> Z versus X -> Z'
    for p in (1 << 34, 2 << 34, 3 << 34):
        assert o.register_alloc(p, 1024) == 0
    o.check_copy(HTOD, 1 << 34, 100, 1024)
    o.check_copy(DTOD, 2 << 34, 1 << 34, 1024)
    o.check_copy(DTOD, 3 << 34, 2 << 34, 1024)
    assert o.read_dev_v(3 << 34, 1024).tobytes() == bytes(v[100:1124])
    o.close()


def pin_records(lib):
    """Records: one per set flag, in (request, flag bit) order, with the
    offsets and counts of the report; strict mode makes undefined
    device-source bytes an error."""
    n_img = 256
    addr = np.ones(n_img, bool)
    addr[10] = False
    v = np.zeros(n_img, np.uint8)
    v[20] = 0x40
    a_bits, vv = _image(addr, v)
    o = O.Oracle(a_bits, vv, lib=lib)
    A, B = 1 << 20, 1 << 21
    assert o.register_alloc(A, 64) == 0
    assert o.register_alloc(B, 64) == 0
    reqs = np.zeros(5, S.REQ_DTYPE)
    reqs[0] = (HTOD, 0, A, 0, 32)       # unaddr at 10, undef at 20
    reqs[1] = (HTOD, 0, A + 58, 0, 8)   # overrun dst, found 6
    reqs[2] = (DTOH, 0, 0, B, 8)        # fresh alloc -> dev undef
    reqs[3] = (DTOD, 0, B + 4, B, 16)   # overlap + dev undef src
    reqs[4] = (DTOD, 0, 77, 99, 5)      # both unallocated
    st, reps, _ = o.check_batch(reqs)
    assert st == 0
    recs = O.emit_records(reps, reqs, strict=False, lib=lib)
    got = [(r["req"], O.FLAG_NAMES[r["cls"]], r["severity"], r["off"], r["count"],
            r["expected"], r["found"]) for r in recs]
    want = [
        (0, "HOST_UNADDR", 0, 10, 1, 32, 31),
        (0, "HOST_UNDEF", 0, 20, 1, 32, 30),
        (1, "OVERRUN_DST", 0, 6, 2, 8, 6),
        (2, "DEV_UNDEF_SRC", 1, 0, 8, 8, 0),
        (3, "DEV_UNDEF_SRC", 1, 0, 16, 16, 0),
        (3, "DTOD_OVERLAP", 1, 4, 12, 16, 0),
        (4, "UNALLOC_DST", 0, 0, 5, 5, 0),
        (4, "UNALLOC_SRC", 0, 0, 5, 5, 0),
    ]
    assert got == want, got
    strict = O.emit_records(reps, reqs, strict=True, lib=lib)
    assert [r["severity"] for r in strict if O.FLAG_NAMES[r["cls"]] == "DEV_UNDEF_SRC"] == [0, 0]
    o.close()


def pin_host_range_errors(lib):
    """Requests outside the host image or of an unknown kind are API errors,
    and a batch holding one is refused before anything runs."""
    a_bits, vv = _image(np.ones(64, bool), np.zeros(64, np.uint8))
    o = O.Oracle(a_bits, vv, lib=lib)
    assert o.register_alloc(1 << 20, 64) == 0
    assert o.check_copy(HTOD, 1 << 20, 60, 8)[0] == -3
    assert o.check_copy(DTOH, (1 << 64) - 1, 1 << 20, 2)[0] == -3
    assert o.check_copy(7, 0, 0, 1)[0] == -2
    reqs = np.zeros(3, S.REQ_DTYPE)
    reqs[0] = (HTOD, 0, 1 << 20, 0, 64)
    reqs[1] = (DTOH, 0, 60, 1 << 20, 8)
    reqs[2] = (HTOD, 0, 1 << 20, 0, 64)
    st, _, bad = o.check_batch(reqs)
    assert st == -3 and bad == 1
    assert np.all(o.read_dev_v(1 << 20, 64) == 0xFF)   # nothing ran
    o.close()


def pin_races(lib):
    """Concurrent accesses (Sec. 2 itemize), scripted traces whose races are
    known by construction: another client's copy still outstanding when
    this one was submitted, one writing what the other reads or writes."""
    R = np.zeros(9, S.REQ_DTYPE)
    # q0 client 0: HtoD writes device [1000, 1100); r1 client 1 DtoH reads
    # device [1050, 1060) while q0 is outstanding -> race with 0
    R[0] = (HTOD, 0, 1000, 0, 100)
    R[1] = (DTOH, 0, 0, 1050, 10)
    # r2 client 1 reads the same device bytes after q0's result -> no race
    R[2] = (DTOH, 0, 0, 1050, 10)
    # r3 client 0 reads device [1020, 1030), which q0 is writing -- but q0
    # is its own client's copy: no race with 0; it writes host [0, 10),
    # which r1 (client 1, still outstanding) also writes -> race with 1
    R[3] = (DTOH, 0, 0, 1020, 10)
    # r4 client 2: HtoD reads host [500, 600), r5 client 3: HtoD reads host
    # [550, 650): two reads -> no race; r5 writes device [7000, 7100), r4
    # writes device [6000, 6100) -> disjoint
    R[4] = (HTOD, 0, 6000, 500, 100)
    R[5] = (HTOD, 0, 7000, 550, 100)
    # r6 client 2: DtoD writes device [7050, 7060) while r5 (client 3)
    # writes [7000, 7100) -> race with 5; its source [1000, 1010) was
    # written by q0 long ago
    R[6] = (DTOD, 0, 7050, 1000, 10)
    # r7 client 1 writes host [0, 10) but did not move data -> never races
    R[7] = (DTOH, 0, 0, 1050, 10)
    # r8 client 3: device [1000, 1100) vs host [1000, 1100): different spaces
    R[8] = (DTOH, 0, 1000, 99999, 10)
    client = np.array([0, 1, 1, 0, 2, 3, 2, 1, 3], np.uint32)
    submit = np.array([10, 20, 200, 30, 300, 310, 320, 330, 340], np.uint64)
    done = np.array([100, 60, 250, 70, 400, 400, 420, 420, 420], np.uint64)
    moved = np.array([1, 1, 1, 1, 1, 1, 1, 0, 1], np.uint8)
    got = O.races(R, client, submit, done, moved, lib=lib)
    assert got.tolist() == [-1, 0, -1, 1, -1, -1, 5, -1, -1], got.tolist()


# ------------------------------------------------ pitched copies, arrays


def _coords(w, h, d):
    """(i, y, z) of every copied byte in the copy's row-major order."""
    z, y, i = np.meshgrid(np.arange(d), np.arange(h), np.arange(w), indexing="ij")
    return i.ravel(), y.ravel(), z.ravel()


def _positions(sd, w, h, d, dims=None):
    """Positions of every copied byte on one side, computed with numpy
    broadcasting: linear memory / host image by pitch and rows, an array by
    its dense (z, y, x) layout."""
    i, y, z = _coords(w, h, d)
    if sd["is_array"]:
        W, H, _ = dims
        return ((sd["z"] + z) * H + sd["y"] + y) * W + sd["x"] + i
    return sd["ptr"] + (sd["z"] + z) * sd["pitch"] * sd["rows"] + (sd["y"] + y) * sd["pitch"] \
        + sd["x"] + i


def pin_strided_footnote(lib):
    """The footnote to Sec. 2's error list: host memory read with a stride is
    not an error.  An array of 24-byte records whose last 8 bytes are
    padding (never written: undefined, some unaddressable) is copied as a
    pitched copy of the 16 payload bytes per record: only the payload is
    classified, with counts and first offsets equal to the payload's class
    list in row-major order; a plain copy of the same span reports the
    padding.  Host->device and device->host (destination A bits)."""
    rng = np.random.default_rng(31)
    rec, pay, nrec = 24, 16, 40
    n_img = rec * nrec + 64
    states = rng.integers(0, len(BYTE_STATES), n_img)
    states[rng.random(n_img) < 0.85] = 4   # mostly (A=1, V=0): good payload
    addr = np.array([BYTE_STATES[k][0] for k in states], bool)
    v = np.array([BYTE_STATES[k][1] for k in states], np.uint8)
    cls = np.array([BYTE_STATES[k][2] for k in states])
    for r_ in range(nrec):  # padding: undefined, every third record unaddressable
        pad = slice(r_ * rec + pay, (r_ + 1) * rec)
        addr[pad] = r_ % 3 != 0
        v[pad] = 0xFF
        cls[pad] = O.BYTE_UNADDR if r_ % 3 == 0 else O.BYTE_UNDEF
    a_bits, vv = _image(addr, v)
    dev = 1 << 40
    for h0 in (0, 5):  # record phase within the image
        for kind in (HTOD, DTOH):
            o = O.Oracle(a_bits, vv, lib=lib)
            assert o.register_alloc(dev, 1 << 16) == 0
            if kind == DTOH:  # a fully defined device source
                assert o.mark(dev, 1 << 16, 0) == 0
            rows = nrec - 1
            hs = O.side(h0, pitch=rec)
            ds = O.side(dev + 100, pitch=pay)
            dst, src = (ds, hs) if kind == HTOD else (hs, ds)
            st, r = o.check_copy3d(kind, dst, src, pay, rows)
            assert st == 0
            payload = [int(cls[h0 + y * rec + i]) for y in range(rows) for i in range(pay)]
            if kind == DTOH:  # the device source is defined: only A matters
                payload = [O.BYTE_UNADDR if c == O.BYTE_UNADDR else O.BYTE_GOOD for c in payload]
            assert _sub(r, SCAN_KEYS) == _expect_from_classes(payload), (h0, kind)
            assert r["expected"] == pay * rows
            # the plain copy of the whole span sees the padding
            span = (rows - 1) * rec + pay
            if kind == HTOD:
                st, r1 = o.check_copy(HTOD, dev + 5000, h0, span)
            else:
                st, r1 = o.check_copy(DTOH, h0, dev, span)
            assert st == 0
            whole = [int(cls[h0 + k]) for k in range(span)]
            if kind == DTOH:
                whole = [O.BYTE_UNADDR if c == O.BYTE_UNADDR else O.BYTE_GOOD for c in whole]
            assert _sub(r1, SCAN_KEYS) == _expect_from_classes(whole)
            assert r1["n_unaddr"] + r1["n_undef"] > r["n_unaddr"] + r["n_undef"]
            o.close()


def pin_pitched_reduces_to_1d(lib, trials: int = 120):
    """Two special cases that are plain copies: contiguous rows and slices
    (pitch = width, rows = height), and a single row (height = depth = 1,
    placed at (z*rows + y)*pitch + x).  Each must give the plain copy's
    report and leave the same shadow state, for every kind."""
    rng = S.rng_for(37)
    n_img = 1 << 13
    v = rng.integers(0, 256, n_img).astype(np.uint8)
    v[rng.random(n_img) < 0.6] = 0
    addr = rng.random(n_img) > 0.1
    a_bits, vv = _image(addr, v)
    d0, d1 = 1 << 36, 1 << 37
    for t in range(trials):
        kind = int(rng.choice([HTOD, DTOH, DTOD]))
        o3, o1 = O.Oracle(a_bits, vv, lib=lib), O.Oracle(a_bits, vv, lib=lib)
        for o in (o3, o1):
            assert o.register_alloc(d0, 4096) == 0 and o.register_alloc(d1, 4096) == 0
            assert o.check_copy(HTOD, d0, 1000, 4096)[0] == 0  # some device state
        if t % 2:
            w, h, d = int(rng.integers(1, 40)), int(rng.integers(1, 6)), int(rng.integers(1, 4))
            n = w * h * d
            sides = [O.side(p, pitch=w, rows=h) for p in (0, 0)]
            offs = []
            for k in range(2):
                dev_side = (k == 0 and kind != DTOH) or (k == 1 and kind != HTOD)
                base = (d0 if k else d1) if dev_side else 0
                lim = 4096 + 64 if dev_side else n_img
                p = base + int(rng.integers(0, lim - n))
                if kind == DTOD and k == 1 and t % 4 == 1:  # overlapping the destination
                    p = int(np.clip(offs[0] + rng.integers(-n, n + 1), d1, d1 + 4096))
                sides[k]["ptr"] = p
                offs.append(p)
        else:
            w, h, d = int(rng.integers(1, 300)), 1, 1
            n = w
            sides, offs = [], []
            for k in range(2):
                dev_side = (k == 0 and kind != DTOH) or (k == 1 and kind != HTOD)
                base = (d0 if k else d1) if dev_side else 0
                pitch, rows = int(rng.integers(0, 50)), int(rng.integers(0, 5))
                x, y, z = int(rng.integers(0, 20)), int(rng.integers(0, 4)), int(rng.integers(0, 3))
                place = (z * rows + y) * pitch + x
                lim = 4096 + 64 if dev_side else n_img - 64
                p = base + int(rng.integers(0, max(1, lim - n - place)))
                sides.append(O.side(p, pitch=pitch, rows=rows, x=x, y=y, z=z))
                offs.append(p + place)
        st3, r3 = o3.check_copy3d(kind, sides[0], sides[1], w, h, d)
        st1, r1 = o1.check_copy(kind, offs[0], offs[1], n)
        assert st3 == st1, (t, st3, st1)
        if st1 == 0:
            assert r3 == r1, (t, kind, r3, r1)
            assert np.array_equal(o3.read_host_v(), o1.read_host_v())
            for b in (d0, d1):
                assert np.array_equal(o3.read_dev_v(b, 4096), o1.read_dev_v(b, 4096))
        o3.close()
        o1.close()


def pin_pitched_bruteforce(lib, trials: int = 150):
    """Random pitched geometry (pitch >= width, rows >= height, origins)
    against formulations that share nothing with the oracle's loops:
    - range: every copied byte's address belongs to the allocation of the
      first one, set membership over the whole extent (R21 asks for the
      extent, first to last copied byte, in one allocation);
    - counts and first offsets: the class of each byte at its numpy-computed
      position, in row-major order;
    - carry: numpy fancy-index assignment (device->device reads the whole
      source first, like memmove);
    - overlap warning: the two spans intersect."""
    rng = S.rng_for(41)
    n_img = 1 << 14
    v = rng.integers(1, 256, n_img).astype(np.uint8)
    v[rng.random(n_img) < 0.7] = 0
    addr = rng.random(n_img) > 0.08
    a_bits, vv = _image(addr, v)
    host_cls = np.where(~addr, O.BYTE_UNADDR, np.where(v != 0, O.BYTE_UNDEF, O.BYTE_GOOD))
    base0 = 1 << 38
    layout = [(0, 3000), (3000, 1000), (5000, 4000)]   # two touching, then a gap
    for t in range(trials):
        kind = int(rng.choice([HTOD, DTOH, DTOD]))
        o = O.Oracle(a_bits, vv, lib=lib)
        dev = np.full(9000, 0xFF, np.uint8)   # model of the modelled device space
        for b, sz in layout:
            assert o.register_alloc(base0 + b, sz) == 0
        o.check_copy(HTOD, base0 + 5000, 2000, 4000)
        dev[5000:9000] = np.where(addr[2000:6000], v[2000:6000], 0xFF)
        w, h, d = int(rng.integers(1, 24)), int(rng.integers(1, 7)), int(rng.integers(1, 4))
        sides = []
        for k in range(2):
            pitch = w + int(rng.integers(0, 20))
            rows = h + int(rng.integers(0, 3))
            x, y, z = (int(rng.integers(0, 8)), int(rng.integers(0, 3)), int(rng.integers(0, 2)))
            dev_side = (k == 0 and kind != DTOH) or (k == 1 and kind != HTOD)
            if dev_side and k == 1 and kind == DTOD and t % 2:  # near the destination
                ptr = int(np.clip(sides[0]["ptr"] + rng.integers(-300, 300), base0, base0 + 8800))
            elif dev_side:
                ptr = base0 + int(rng.integers(0, 8800))
            else:
                ptr = int(rng.integers(0, n_img // 2))
            sides.append(O.side(ptr, pitch=pitch, rows=rows, x=x, y=y, z=z))
        st, r = o.check_copy3d(kind, sides[0], sides[1], w, h, d)
        assert st == 0, (t, st)
        pos = [_positions(sd, w, h, d) for sd in sides]
        ok = {}
        for k, name in ((0, "DST"), (1, "SRC")):
            dev_side = (k == 0 and kind != DTOH) or (k == 1 and kind != HTOD)
            if not dev_side:
                continue
            rel = pos[k] - base0
            first = int(rel[0])
            own = _owner(layout, first)
            lo, hi = first, first + int(rel.max() - rel.min()) + 1  # the extent
            if own is None:
                want = "UNALLOC"
            else:
                want = "OK" if all(_owner(layout, a) == own for a in range(lo, hi)) else "OVERRUN"
            got = "UNALLOC" if r["flags"] & F["UNALLOC_" + name] else \
                "OVERRUN" if r["flags"] & F["OVERRUN_" + name] else "OK"
            assert got == want, (t, name, got, want)
            ok[k] = want == "OK"
        # classes
        if kind == HTOD:
            c = host_cls[pos[1]]
        elif kind == DTOH:
            c = np.where(~addr[pos[0]], O.BYTE_UNADDR, O.BYTE_GOOD)
            if ok[1]:
                c = np.where((c == O.BYTE_GOOD) & (dev[pos[1] - base0] != 0), O.BYTE_UNDEF, c)
        else:
            c = np.full(w * h * d, O.BYTE_GOOD)
            if ok[1]:
                c = np.where(dev[pos[1] - base0] != 0, O.BYTE_UNDEF, O.BYTE_GOOD)
        assert _sub(r, SCAN_KEYS) == _expect_from_classes([int(x) for x in c]), (t, kind)
        if kind == DTOD:
            sp = [(int(p.min()), int(p.max()) + 1) for p in pos]
            inter = sp[0][0] < sp[1][1] and sp[1][0] < sp[0][1]
            assert bool(r["flags"] & F["DTOD_OVERLAP"]) == inter, t
        # carry
        hv = v.copy()
        if kind == HTOD and ok[0]:
            dev[pos[0] - base0] = np.where(addr[pos[1]], v[pos[1]], 0xFF)
        elif kind == DTOH and ok[1]:
            src_v = dev[pos[1] - base0]
            m = addr[pos[0]]
            hv[pos[0][m]] = src_v[m]
        elif kind == DTOD and ok[0] and ok[1]:
            tmp = dev[pos[1] - base0].copy()
            dev[pos[0] - base0] = tmp
        assert np.array_equal(o.read_host_v(), hv), (t, kind)
        for b, sz in layout:
            got = o.read_dev_v(base0 + b, sz)
            assert np.array_equal(got, dev[b:b + sz]), (t, kind, b)
        o.close()


def pin_arrays(lib):
    """Device arrays (Fig. 2's second list): keyed by handle, bounds checked
    per dimension, dense row-major shadow.  Checked against numpy block
    assignment on a (D, H, W) array and enumeration of the copied box."""
    rng = S.rng_for(43)
    n_img = 1 << 13
    v = rng.integers(0, 256, n_img).astype(np.uint8)
    v[rng.random(n_img) < 0.5] = 0
    addr = rng.random(n_img) > 0.05
    a_bits, vv = _image(addr, v)
    W, H, D = 40, 12, 5
    A1, A2 = 0x1000, 0x2000           # handles: a namespace of their own
    o = O.Oracle(a_bits, vv, lib=lib)
    assert o.register_array(A1, W, H, D) == 0
    assert o.register_array(A2, 16, 16, 1) == 0
    assert o.register_array(A1, 4, 4, 1) == O.STATUS_CODES["E_OVERLAP"]
    assert o.register_array(0x3000, 0, 4, 1) == O.STATUS_CODES["E_ZERO_SIZE"]
    assert o.register_alloc(A1, 64) == 0   # the same number as an address: no clash
    model = np.full((D, H, W), 0xFF, np.uint8)
    assert np.array_equal(o.read_array_v(A1, 0, W * H * D), model.ravel())
    for t in range(150):
        x, y, z = int(rng.integers(0, W)), int(rng.integers(0, H)), int(rng.integers(0, D))
        if t % 4:  # mostly boxes that fit, some reaching the far faces exactly
            w, h, d = (int(rng.integers(1, W - x + 1)), int(rng.integers(1, H - y + 1)),
                       int(rng.integers(1, D - z + 1)))
        else:
            w, h, d = (int(rng.integers(1, W + 4)), int(rng.integers(1, H + 3)),
                       int(rng.integers(1, D + 2)))
        fits = all(0 <= c < lim for (c, lim) in
                   [(x + w - 1, W), (y + h - 1, H), (z + d - 1, D)])
        kind = int(rng.choice([HTOD, DTOH, DTOD]))
        arr = O.side(A1, x=x, y=y, z=z, array=True)
        hp = int(rng.integers(w, w + 30))
        hrows = h + int(rng.integers(0, 3))
        host = O.side(int(rng.integers(0, 2000)), pitch=hp, rows=hrows)
        hv = o.read_host_v()   # device->host copies change it
        if kind == HTOD:
            st, r = o.check_copy3d(HTOD, arr, host, w, h, d)
            flag = "DST"
        elif kind == DTOH:
            st, r = o.check_copy3d(DTOH, host, arr, w, h, d)
            flag = "SRC"
        else:  # array -> itself at another origin
            x2, y2, z2 = (int(rng.integers(0, W - w + 1)) if w <= W else 0,
                          int(rng.integers(0, H - h + 1)) if h <= H else 0,
                          int(rng.integers(0, D - d + 1)) if d <= D else 0)
            fits2 = x2 + w <= W and y2 + h <= H and z2 + d <= D
            st, r = o.check_copy3d(DTOD, O.side(A1, x=x2, y=y2, z=z2, array=True), arr, w, h, d)
            flag = "SRC"
        assert st == 0, (t, st)
        assert bool(r["flags"] & F["OVERRUN_" + flag]) == (not fits), (t, x, y, z, w, h, d)
        assert r["alloc_base_" + flag.lower()] == A1 and r["alloc_size_" + flag.lower()] == W * H * D
        assert r["found_" + flag.lower()] == W * H * D - ((z * H + y) * W + x)
        hpos = _positions(host, w, h, d)
        if kind == HTOD and fits:
            blk = np.where(addr[hpos], hv[hpos], 0xFF).reshape(d, h, w)
            model[z:z + d, y:y + h, x:x + w] = blk
            assert r["n_unaddr"] == int((~addr[hpos]).sum())
        elif kind == DTOH:
            exp_undef = int(((model[z:z + d, y:y + h, x:x + w].ravel() != 0) & addr[hpos]).sum()) \
                if fits else 0
            assert r["n_undef"] == exp_undef, t
            if fits:
                src = model[z:z + d, y:y + h, x:x + w].ravel()
                cur = o.read_host_v()
                assert np.array_equal(cur[hpos[addr[hpos]]], src[addr[hpos]])
        elif kind == DTOD:
            assert bool(r["flags"] & F["OVERRUN_DST"]) == (not fits2)
            if fits and fits2:
                tmp = model[z:z + d, y:y + h, x:x + w].copy()
                model[z2:z2 + d, y2:y2 + h, x2:x2 + w] = tmp
                a0 = (z * H + y) * W + x
                b0 = (z2 * H + y2) * W + x2
                span = ((d - 1) * H + (h - 1)) * W + w
                assert bool(r["flags"] & F["DTOD_OVERLAP"]) == (a0 < b0 + span and b0 < a0 + span)
        assert np.array_equal(o.read_array_v(A1, 0, W * H * D), model.ravel()), (t, kind)
    # array <-> linear memory, both ways
    assert o.check_copy3d(DTOD, O.side(A1 + 0, pitch=8, rows=2), O.side(A2, x=3, y=1, array=True),
                          8, 2, 1)[0] == 0
    # an unknown handle is unallocated; the host side is never an array
    st, r = o.check_copy3d(HTOD, O.side(0x9999, array=True), O.side(0, pitch=4), 4, 1)
    assert st == 0 and r["flags"] & F["UNALLOC_DST"] and r["found_dst"] == 0
    assert o.check_copy3d(HTOD, O.side(A2, array=True), O.side(A1, array=True), 4, 1)[0] == \
        O.STATUS_CODES["E_ARG"]
    # destroy: ok, then double; unknown; re-creation clears the freed mark
    assert o.free_array(A2) == "OK" and o.free_array(A2) == "DOUBLE"
    assert o.free_array(0x7777) == "UNKNOWN"
    st, r = o.check_copy3d(HTOD, O.side(A2, array=True), O.side(0, pitch=4), 4, 1)
    assert r["flags"] & F["UNALLOC_DST"]
    assert o.register_array(A2, 8, 8, 1) == 0 and o.free_array(A2) == "OK"
    o.close()


def pin_pitched_args(lib):
    """Argument rules of pitched copies: rows closer than the width, slices
    closer than the rows, a host span outside the image, an empty copy (no
    range check at all, R9) and 64-bit overflow of the geometry."""
    a_bits, vv = _image(np.ones(256, bool), np.zeros(256, np.uint8))
    o = O.Oracle(a_bits, vv, lib=lib)
    dev = 1 << 30
    assert o.register_alloc(dev, 4096) == 0
    E = O.STATUS_CODES
    ok = lambda st: st == 0  # noqa: E731
    assert o.check_copy3d(HTOD, O.side(dev, pitch=7), O.side(0, pitch=8), 8, 2)[0] == E["E_ARG"]
    assert o.check_copy3d(HTOD, O.side(dev, pitch=8), O.side(0, pitch=7), 8, 2)[0] == E["E_ARG"]
    assert ok(o.check_copy3d(HTOD, O.side(dev, pitch=0), O.side(0, pitch=0), 8, 1)[0])
    assert o.check_copy3d(HTOD, O.side(dev, pitch=8, rows=1), O.side(0, pitch=8, rows=2),
                          8, 2, 2)[0] == E["E_ARG"]
    assert ok(o.check_copy3d(HTOD, O.side(dev, pitch=8, rows=2), O.side(0, pitch=8, rows=2),
                             8, 2, 2)[0])
    # host span: rows 0..3 of pitch 64 end at 3*64+16 = 208 <= 256; one more row does not
    assert ok(o.check_copy3d(HTOD, O.side(dev, pitch=16), O.side(0, pitch=64), 16, 4)[0])
    assert o.check_copy3d(HTOD, O.side(dev, pitch=16), O.side(0, pitch=64), 16, 5)[0] == \
        E["E_HOST_RANGE"]
    assert o.check_copy3d(DTOH, O.side(200, pitch=64), O.side(dev, pitch=16), 16, 1)[0] == 0
    assert o.check_copy3d(DTOH, O.side(0, pitch=64, y=3), O.side(dev, pitch=16), 65, 1)[0] == \
        E["E_HOST_RANGE"]
    # empty copies: nothing is checked
    for whd in ((0, 5, 5), (5, 0, 5), (5, 5, 0)):
        st, r = o.check_copy3d(HTOD, O.side(12345, array=True), O.side(10**12), *whd)
        assert st == 0 and r["flags"] == 0 and r["expected"] == 0 and r["first_bad_off"] == -1
    # the extent of the last row ends exactly at the allocation's end
    st, r = o.check_copy3d(HTOD, O.side(dev + 4096 - (3 * 100 + 10), pitch=100), O.side(0, pitch=10),
                           10, 4)
    assert st == 0 and r["flags"] == 0 and r["found_dst"] == 3 * 100 + 10
    st, r = o.check_copy3d(HTOD, O.side(dev + 4096 - (3 * 100 + 9), pitch=100), O.side(0, pitch=10),
                           10, 4)
    assert r["flags"] & F["OVERRUN_DST"] and r["found_dst"] == 3 * 100 + 9
    # slices: the extent uses rows per slice, not height
    st, r = o.check_copy3d(HTOD, O.side(dev, pitch=10, rows=100), O.side(0, pitch=10, rows=3),
                           10, 3, 5)
    assert st == 0 and r["flags"] == 0
    st, r = o.check_copy3d(HTOD, O.side(dev, pitch=10, rows=100), O.side(0, pitch=10, rows=3),
                           10, 3, 6)
    assert r["flags"] & F["OVERRUN_DST"] and r["found_dst"] == 4096
    # geometry beyond 64 bits
    big = 1 << 62
    assert o.check_copy3d(HTOD, O.side(dev, pitch=big, rows=8), O.side(0, pitch=8, rows=8),
                          8, 2, 2)[0] == E["E_WRAP"]
    o.close()


# ------------------------------------------------ memset, kernel arguments


def pin_memset(lib, trials: int = 200):
    """Memset wrappers: the range verdict equals set membership over the
    extent; with a valid range exactly the written bytes become defined
    (numpy model of the device space), nothing else changes; a failed range
    changes nothing; a later device->host copy of the written bytes finds
    them defined.  Argument rules: rows closer than the width, overflow,
    empty memsets."""
    rng = S.rng_for(53)
    n_img = 1 << 14
    a_bits, vv = _image(np.ones(n_img, bool), rng.integers(0, 256, n_img).astype(np.uint8))
    base0 = 1 << 39
    layout = [(0, 3000), (3000, 1000), (5000, 4000)]
    o = O.Oracle(a_bits, vv, lib=lib)
    dev = np.full(9000, 0xFF, np.uint8)
    for b, sz in layout:
        assert o.register_alloc(base0 + b, sz) == 0
    o.check_copy(HTOD, base0 + 5000, 100, 4000)
    dev[5000:9000] = vv[100:4100]
    for t in range(trials):
        w, h = int(rng.integers(1, 200)), int(rng.integers(1, 8))
        pitch = w + int(rng.integers(0, 100)) if h > 1 else int(rng.integers(0, 300))
        d = int(rng.integers(0, 9000))
        st, r = o.memset(base0 + d, w, h, pitch)
        assert st == 0
        ext = (h - 1) * pitch + w
        own = _owner(layout, d)
        want = "UNALLOC" if own is None else \
            "OK" if all(_owner(layout, a) == own for a in range(d, d + ext)) else "OVERRUN"
        got = "UNALLOC" if r["flags"] & F["UNALLOC_DST"] else \
            "OVERRUN" if r["flags"] & F["OVERRUN_DST"] else "OK"
        assert got == want, (t, d, w, h, pitch, got, want)
        assert r["expected"] == r["n_good"] == w * h and r["n_undef"] == r["n_unaddr"] == 0
        if want == "OK":
            rows = (d + np.arange(h)[:, None] * pitch + np.arange(w)[None, :]).ravel()
            dev[rows] = 0
        for b, sz in layout:
            assert np.array_equal(o.read_dev_v(base0 + b, sz), dev[b:b + sz]), (t, b)
    # a memset region copied back to the host is defined
    st, _ = o.memset(base0 + 100, 64, 1)
    st, r = o.check_copy(DTOH, 0, base0 + 100, 64)
    assert st == 0 and r["n_undef"] == 0
    E = O.STATUS_CODES
    assert o.memset(base0, 10, 2, 9)[0] == E["E_ARG"]
    assert o.memset(base0, 10, 1, 0)[0] == 0
    assert o.memset(base0, 1 << 40, 1 << 30, 1 << 40)[0] == E["E_WRAP"]
    st, r = o.memset(12345, 0, 7)
    assert st == 0 and r["flags"] == 0 and r["expected"] == 0
    o.close()
    # carry off: verdicts only
    o = O.Oracle(a_bits, vv, carry=False, lib=lib)
    assert o.register_alloc(base0, 100) == 0
    st, r = o.memset(base0, 100)
    assert st == 0 and r["flags"] == 0
    assert np.all(o.read_dev_v(base0, 100) == 0xFF)
    o.close()


def pin_kernel_args(lib, trials: int = 120):
    """Kernel arguments: range verdicts by set membership (a zero extent:
    containment of the pointer alone); undefined bytes of a read argument
    counted against the device model, first offset relative to the
    pointer; every read sees the state before the launch (an argument
    written and read in the same launch still reports what was undefined);
    afterwards exactly the valid write ranges are defined.  Access values
    outside read/write are refused with nothing changed."""
    rng = S.rng_for(59)
    n_img = 1 << 14
    v = rng.integers(0, 256, n_img).astype(np.uint8)
    v[rng.random(n_img) < 0.6] = 0
    a_bits, vv = _image(np.ones(n_img, bool), v)
    base0 = 1 << 41
    layout = [(0, 3000), (3000, 1000), (5000, 4000)]
    R, W = O.ARG_READ, O.ARG_WRITE
    o = O.Oracle(a_bits, vv, lib=lib)
    dev = np.full(9000, 0xFF, np.uint8)
    for b, sz in layout:
        assert o.register_alloc(base0 + b, sz) == 0
    o.check_copy(HTOD, base0 + 200, 0, 2800)
    dev[200:3000] = v[:2800]
    o.check_copy(HTOD, base0 + 5000, 4000, 4000)
    dev[5000:9000] = v[4000:8000]
    for t in range(trials):
        k = int(rng.integers(1, 6))
        ptr = [int(rng.integers(0, 9100)) for _ in range(k)]
        if t % 3 == 0 and k > 1:
            ptr[1] = ptr[0]     # aliasing arguments
        nb = [int(rng.integers(0, 800)) if rng.random() > 0.1 else 0 for _ in range(k)]
        acc = [int(rng.choice([R, W, R | W])) for _ in range(k)]
        st, reps = o.check_kernel_args([base0 + p for p in ptr], nb, acc)
        assert st == 0
        after = dev.copy()
        for i in range(k):
            r = reps[i]
            own = _owner(layout, ptr[i])
            if own is None:
                want = "UNALLOC"
            elif all(_owner(layout, a) == own for a in range(ptr[i], ptr[i] + nb[i])):
                want = "OK"
            else:
                want = "OVERRUN"
            for side, bit in (("SRC", R), ("DST", W)):
                got = "UNALLOC" if r["flags"] & F["UNALLOC_" + side] else \
                    "OVERRUN" if r["flags"] & F["OVERRUN_" + side] else "OK"
                assert got == (want if acc[i] & bit else "OK"), (t, i, side, got, want)
            assert r["expected"] == nb[i]
            if acc[i] & R and want == "OK":
                seg = dev[ptr[i]:ptr[i] + nb[i]]          # the state before the launch
                bad = np.nonzero(seg != 0)[0]
                assert r["n_undef"] == bad.size and r["n_good"] == nb[i] - bad.size
                assert r["first_undef_off"] == (int(bad[0]) if bad.size else -1)
                assert bool(r["flags"] & F["DEV_UNDEF_SRC"]) == bool(bad.size)
            else:
                assert r["n_undef"] == 0 and not r["flags"] & F["DEV_UNDEF_SRC"]
            if acc[i] & W and want == "OK":
                after[ptr[i]:ptr[i] + nb[i]] = 0
        dev = after
        for b, sz in layout:
            assert np.array_equal(o.read_dev_v(base0 + b, sz), dev[b:b + sz]), (t, b)
    # refused as a whole: nothing changes
    before = o.read_dev_v(base0, 3000).copy()
    st, _ = o.check_kernel_args([base0, base0], [100, 100], [W, 4])
    assert st == O.STATUS_CODES["E_ARG"]
    st, _ = o.check_kernel_args([base0], [100], [0])
    assert st == O.STATUS_CODES["E_ARG"]
    assert np.array_equal(o.read_dev_v(base0, 3000), before)
    o.close()


ALL_PINS = [
    pin_listing5, pin_htod_bytes_by_construction, pin_dtoh_bytes_by_construction,
    pin_range_bruteforce, pin_free_sequences, pin_free_sequences_reuse, pin_generator_truth,
    pin_invariants, pin_carry_roundtrip, pin_mark, pin_dtod_memmove, pin_records,
    pin_host_range_errors, pin_races, pin_strided_footnote, pin_pitched_reduces_to_1d,
    pin_pitched_bruteforce, pin_arrays, pin_pitched_args, pin_memset, pin_kernel_args,
]


def run_all(lib_path: str | None = None) -> list[str]:
    """Run every pin; return the names of those that failed."""
    lib = O.load(lib_path)
    failed = []
    for p in ALL_PINS:
        try:
            p(lib)
        except AssertionError:
            failed.append(p.__name__)
    return failed


if __name__ == "__main__":
    bad = run_all(sys.argv[1] if len(sys.argv) > 1 else None)
    print("FAILED:" + ",".join(bad) if bad else "ALL PINS PASS")
    sys.exit(1 if bad else 0)

"""GPU parity: libcg (through its C ABI) against the CPU oracle, bit-exact.

Every verdict is an integer, so the tolerance is zero: reports, records and
the final host/device V shadow must equal the oracle's."""
from __future__ import annotations

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


def _run_single(ctx, orc, reqs, what):
    reports = []
    for i, q in enumerate(reqs):
        k, d, s, n = int(q["kind"]), int(q["dst"]), int(q["src"]), int(q["n"])
        st_g, g = ctx.check_copy(k, d, s, n)
        st_o, o = orc.check_copy(k, d, s, n)
        assert st_g == st_o == 0, (what, i, st_g, st_o)
        U.assert_same_report(g, o, f"{what} request {i} {q}")
        reports.append(o)
    return reports


ENGINES = {"regs": 1, "tma": 2}


@pytest.mark.parametrize("engine", sorted(ENGINES))
@pytest.mark.parametrize("carry", [True, False])
def test_small_workload_single_checks(cg, carry, engine):
    """1,000 mixed copies over 64 live allocations, one cg_check_copy each."""
    w = S.small(0)
    ctx, orc, (a, v) = U.make_pair(w.image, w.table, carry=carry, scan_engine=ENGINES[engine])
    _run_single(ctx, orc, w.reqs, "small/single")
    U.assert_same_state(ctx, orc, v, w.table)


@pytest.mark.parametrize("engine", sorted(ENGINES))
@pytest.mark.parametrize("seed", [0, 1])
@pytest.mark.parametrize("seg_kib", [2, 64])
def test_small_workload_batch(cg, seed, seg_kib, engine):
    """The same stream as one cg_check_batch: reports, records (order and
    content) and final state equal the oracle's sequential result."""
    w = S.small(seed)
    ctx, orc, (a, v) = U.make_pair(w.image, w.table, batch_segment_kib=seg_kib,
                                   scan_engine=ENGINES[engine])
    st, reps, recs, total, _ = ctx.check_batch(w.reqs)
    assert st == 0, cg.cg_last_error()
    st_o, oreps, _ = orc.check_batch(w.reqs)
    assert st_o == 0
    for i, (g, o) in enumerate(zip(U.reports_from_array(reps), oreps)):
        U.assert_same_report(g, o, f"batch request {i}")
    orecs = O.emit_records(oreps, w.reqs)
    assert total == len(orecs)
    assert U.reports_from_array(recs) == orecs
    U.assert_same_state(ctx, orc, v, w.table)
    assert ctx.stats()["levels"] >= 1


def test_batch_equals_single(cg):
    """Each report of a batch equals the same copy checked alone in order."""
    w = S.small(2)
    c1, _, (a1, v1) = U.make_pair(w.image, w.table)
    c2, _, (a2, v2) = U.make_pair(w.image, w.table)
    st, reps, _, _, _ = c1.check_batch(w.reqs)
    assert st == 0
    for i, q in enumerate(w.reqs):
        st, g = c2.check_copy(int(q["kind"]), int(q["dst"]), int(q["src"]), int(q["n"]))
        assert st == 0
        U.assert_same_report(U.reports_from_array(reps[i:i + 1])[0], g, f"request {i}")
    assert np.array_equal(v1.cpu().numpy(), v2.cpu().numpy())


def _mixed_image(n, seed):
    rng = np.random.default_rng(seed)
    v = rng.integers(0, 256, n).astype(np.uint8)
    v[rng.random(n) < 0.6] = 0
    addr = rng.random(n) > 0.15
    return S.HostImage(S.pack_a(addr), v, [], None)


@pytest.mark.parametrize("engine", sorted(ENGINES))
@pytest.mark.parametrize("kind", [HTOD, DTOH, DTOD])
def test_alignment_sweep(cg, kind, engine):
    """Every host offset mod 16 against every device offset mod 16, sizes
    around the 16-byte vector, the 512-byte warp row, the 2 KiB step and the
    4 KiB TMA tile."""
    img = _mixed_image(1 << 16, 5)
    base = 1 << 40
    table = S.AllocTable(np.array([base, base + (1 << 20)], np.uint64),
                         np.array([1 << 18, 1 << 18], np.uint64), np.zeros(0, np.int64))
    ctx, orc, (a, v) = U.make_pair(img, table, scan_engine=ENGINES[engine])
    # give the device shadows mixed content first
    for off in range(0, 1 << 18, 1 << 15):
        for b in (base, base + (1 << 20)):
            assert ctx.check_copy(HTOD, b + off, off % (1 << 15), 1 << 15)[0] == 0
            orc.check_copy(HTOD, b + off, off % (1 << 15), 1 << 15)
    sizes = [1, 2, 15, 16, 17, 31, 33, 100, 511, 512, 513, 2047, 2048, 2049, 4095, 4096,
             4097, 5000, 8193, 20000]
    rng = np.random.default_rng(kind)
    reqs = []
    for ho in range(16):
        for do in range(16):
            n = sizes[(ho * 16 + do) % len(sizes)]
            h = int(rng.integers(0, 1000)) * 16 + ho
            dv = base + int(rng.integers(0, 1000)) * 16 + do
            if kind == HTOD:
                reqs.append((kind, 0, dv, h, n))
            elif kind == DTOH:
                reqs.append((kind, 0, h, dv, n))
            else:
                reqs.append((kind, 0, base + (1 << 20) + int(rng.integers(0, 1000)) * 16 + ho,
                             dv, n))
    reqs = np.array(reqs, dtype=S.REQ_DTYPE)
    _run_single(ctx, orc, reqs, "sweep")
    U.assert_same_state(ctx, orc, v, table)
    # the same requests again as one batch, on fresh state
    ctx2, orc2, (a2, v2) = U.make_pair(img, table, scan_engine=ENGINES[engine])
    st, reps, recs, total, _ = ctx2.check_batch(reqs)
    st_o, oreps, _ = orc2.check_batch(reqs)
    assert st == st_o == 0
    for i, (g, o) in enumerate(zip(U.reports_from_array(reps), oreps)):
        U.assert_same_report(g, o, f"sweep batch {i}")
    U.assert_same_state(ctx2, orc2, v2, table)


@pytest.mark.parametrize("engine", sorted(ENGINES))
def test_edge_cases(cg, engine):
    """Empty copies, wild and wrapping pointers, API errors, frees."""
    img = _mixed_image(8192, 1)
    base = 1 << 30
    table = S.AllocTable(np.array([base, base + 4096], np.uint64),
                         np.array([4096, 256], np.uint64), np.zeros(0, np.int64))
    ctx, orc, (a, v) = U.make_pair(img, table, scan_engine=ENGINES[engine])
    cases = [
        (HTOD, base, 0, 0), (DTOH, 0, 12345, 0), (DTOD, 1, 2, 0),           # n == 0
        (HTOD, base + 4096 - 1, 10, 1), (HTOD, base + 4095, 10, 2),          # last byte / overrun
        (HTOD, base + 4096 + 256, 0, 1),                                      # one past the table
        (HTOD, (1 << 64) - 16, 0, 64),                                        # wild, would wrap
        (DTOH, 0, base, 4096 + 256),                                          # spans two allocations
        (DTOD, base + 4096, base, 256), (DTOD, base, base + 1, 300),          # overlap, memmove
        (DTOD, base + 100, base + 90, 50), (DTOD, 5, 7, 3),
        (HTOD, base, 4096 - 7, 7),
    ]
    for i, (k, d, s, n) in enumerate(cases):
        st_g, g = ctx.check_copy(k, d, s, n)
        st_o, o = orc.check_copy(k, d, s, n)
        assert st_g == st_o == 0, (i, st_g, st_o)
        U.assert_same_report(g, o, f"edge case {i}")
    U.assert_same_state(ctx, orc, v, table)
    # API errors leave everything untouched
    assert ctx.check_copy(HTOD, base, 8190, 8)[0] == -3
    assert ctx.check_copy(DTOH, 8191, base, 2)[0] == -3
    assert ctx.check_copy(9, 0, 0, 1)[0] == -2
    reqs = np.array([(HTOD, 0, base, 0, 16), (DTOH, 0, 8191, base, 2)], dtype=S.REQ_DTYPE)
    st, _, _, _, bad = ctx.check_batch(reqs)
    assert st == -3 and bad == 1
    U.assert_same_state(ctx, orc, v, table)
    # registration errors and free verdicts
    assert ctx.register_alloc(base + 10, 10) == -6
    assert ctx.register_alloc(7, 0) == -4
    assert ctx.register_alloc((1 << 64) - 8, 16) == -5
    assert ctx.free(base + 10) == "INTERIOR"
    assert ctx.free(base + 4096) == "OK"
    assert ctx.free(base + 4096) == "DOUBLE"
    assert ctx.free(99) == "UNKNOWN"
    # mark defined / undefined (client requests)
    assert ctx.mark_defined(base + 100, 50) == 0
    assert orc.mark(base + 100, 50, 0) == 0
    assert ctx.mark_undefined(base + 120, 10) == 0
    assert orc.mark(base + 120, 10, 0xFF) == 0
    assert ctx.mark_defined(base + 4000, 200) == -8
    st_g, g = ctx.check_copy(DTOH, 0, base + 90, 100)
    st_o, o = orc.check_copy(DTOH, 0, base + 90, 100)
    U.assert_same_report(g, o, "after mark")


def test_no_image_bound(cg):
    ctx = cg.Context()
    assert ctx.register_alloc(1 << 20, 64) == 0
    assert ctx.check_copy(HTOD, 1 << 20, 0, 8)[0] == -10
    st, r = ctx.check_copy(DTOD, 1 << 20, (1 << 20) + 8, 16)
    assert st == 0 and r["flags"] == cg.FLAGS["DEV_UNDEF_SRC"] | cg.FLAGS["DTOD_OVERLAP"]
    st, r = ctx.check_copy(DTOD, 1 << 20, (1 << 20) + 8, 8)   # touching, not overlapping
    assert st == 0 and r["flags"] == cg.FLAGS["DEV_UNDEF_SRC"]


@pytest.mark.parametrize("strict", [False, True])
def test_adversarial_density(cg, strict):
    """Half the bytes undefined with partial masks, 5 % unaddressable: every
    copy reports; records compacted in (request, class) order."""
    w = S.adversarial(3, n_req=400, host_n=32 << 20, n_alloc=256)
    # keep the copies small enough for the oracle to be quick
    w.reqs["n"] = np.minimum(w.reqs["n"], 1 << 20)
    for q in w.reqs:
        if q["kind"] == HTOD:
            q["src"] = min(int(q["src"]), w.image.n - int(q["n"]))
        elif q["kind"] == DTOH:
            q["dst"] = min(int(q["dst"]), w.image.n - int(q["n"]))
    ctx, orc, (a, v) = U.make_pair(w.image, w.table, strict=strict)
    st, reps, recs, total, _ = ctx.check_batch(w.reqs)
    assert st == 0
    st_o, oreps, _ = orc.check_batch(w.reqs)
    for i, (g, o) in enumerate(zip(U.reports_from_array(reps), oreps)):
        U.assert_same_report(g, o, f"adversarial {i}")
    orecs = O.emit_records(oreps, w.reqs, strict=strict)
    assert total == len(orecs) and U.reports_from_array(recs) == orecs
    assert all(r["flags"] for r in oreps)
    U.assert_same_state(ctx, orc, v, w.table)
    # truncated record buffer: the first rec_cap records, full count
    ctx2, _, _ = U.make_pair(w.image, w.table, strict=strict)
    st, _, recs2, total2, _ = ctx2.check_batch(w.reqs, rec_cap=17)
    assert st == 0 and total2 == total
    assert U.reports_from_array(recs2) == orecs[:17]


def test_large_table_batch(cg):
    """A 1,000,000-entry allocation table: the device lookup (splitters in
    shared memory) gives the oracle's range verdicts for every request."""
    rng = S.rng_for(4)
    table = S.alloc_table(rng, 1_000_000, 256, 64 << 10, log_sizes=True)
    img = S.host_image_runs(rng, 16 << 20, 1e-4, 8.0, 0.5, 1e-5)
    reqs = S.requests(rng, 3000, table, img.n, 16, 256 << 10, p_wild=0.02)
    ctx, orc, (a, v) = U.make_pair(img, table)
    st, reps, recs, total, _ = ctx.check_batch(reqs)
    assert st == 0
    st_o, oreps, _ = orc.check_batch(reqs)
    for i, (g, o) in enumerate(zip(U.reports_from_array(reps), oreps)):
        U.assert_same_report(g, o, f"large-table {i}")
    orecs = O.emit_records(oreps, reqs)
    assert total == len(orecs) and U.reports_from_array(recs) == orecs
    gv = v.cpu().numpy()
    assert np.array_equal(gv, orc.read_host_v())


def test_host_resident_image(cg):
    """An image in pinned host memory is read in place (register engine);
    results equal the oracle's.  Pageable host memory is refused."""
    import torch
    w = S.small(6)
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
    _run_single(ctx, orc, w.reqs[:400], "host image/single")
    st, reps, _, _, _ = ctx.check_batch(w.reqs[400:])
    st_o, oreps, _ = orc.check_batch(w.reqs[400:])
    assert st == st_o == 0
    for i, (g, o) in enumerate(zip(U.reports_from_array(reps), oreps)):
        U.assert_same_report(g, o, f"host image/batch {i}")
    torch.cuda.synchronize()
    assert np.array_equal(v_h.numpy(), orc.read_host_v())
    pageable = torch.zeros(n, dtype=torch.uint8)
    st = cg.cg_bind_host_shadow(ctx.handle, a_h.data_ptr(), pageable.data_ptr(), n)
    assert st == -1

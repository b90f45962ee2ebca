"""Table updates on the device: after the first upload, registrations and
frees reach the device copy of the allocation table through the merge
kernel (no whole-table upload).  The device table equals the sorted list
of live allocations after every round of events, entries that stay keep
their shadow address, and batches checked against it give the oracle's
reports (copies into freed and re-registered allocations included)."""
from __future__ import annotations

import random

import numpy as np
import pytest

import cg_synth as S
from tests import gpu_util as U

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cg():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1310_0901_gb300 as m
    return m


def _live_sorted(live: dict) -> tuple[np.ndarray, np.ndarray]:
    b = np.array(sorted(live), dtype=np.uint64)
    return b, np.array([live[int(x)] for x in b], dtype=np.uint64)


def _events(rng, live, freed, ctx, orc, n_free, n_new, n_reuse):
    """Free n_free live allocations; register n_new fresh ones above 2^48 and
    n_reuse at the bases of allocations freed in this round (smaller)."""
    gone = rng.sample(sorted(live), min(n_free, len(live)))
    for b in gone:
        assert ctx.free(b) == orc.free(b) == "OK"
        freed[b] = live.pop(b)
    top = max([b + s for b, s in live.items()] + [1 << 48])
    for k in range(n_new):
        b = ((top + 4096) & ~255) + k * (1 << 20)
        s = rng.randrange(1, 1 << 19)
        assert ctx.register_alloc(b, s) == orc.register_alloc(b, s) == 0
        live[b] = s
    for b in gone[:n_reuse]:
        s = max(1, freed[b] // 2)
        assert ctx.register_alloc(b, s) == orc.register_alloc(b, s) == 0
        live[b] = s


@pytest.mark.parametrize("seed", [0, 1])
def test_device_table_follows_events_through_merges(cg, seed):
    rng = random.Random(seed)
    w = S.small(seed)
    ctx, orc, (a, v) = U.make_pair(w.image, w.table)
    freed_j = set(int(j) for j in w.table.freed)
    live = {int(w.table.base[j]): int(w.table.size[j]) for j in range(len(w.table.base))
            if j not in freed_j}
    freed = {}
    base0, size0, sh0 = ctx.device_table()
    want_b, want_s = _live_sorted(live)
    assert np.array_equal(base0, want_b) and np.array_equal(size0, want_s)
    uploads = ctx.stats()["table_uploads"]
    assert uploads == 1 and ctx.stats()["table_merges"] == 0
    shadow_of = dict(zip(base0.tolist(), sh0.tolist()))
    parts = np.array_split(w.reqs, 5)
    for rnd, p in enumerate(parts):
        _events(rng, live, freed, ctx, orc, n_free=rng.randrange(0, 9),
                n_new=rng.randrange(0, 6), n_reuse=rng.randrange(0, 3))
        st, reps, _, _, _ = ctx.check_batch(p)
        st_o, oreps, _ = orc.check_batch(p)
        assert st == st_o == 0
        for i, (g, o) in enumerate(zip(U.reports_from_array(reps), oreps)):
            U.assert_same_report(g, o, f"round {rnd} request {i}")
        b, s, sh = ctx.device_table()
        want_b, want_s = _live_sorted(live)
        assert np.array_equal(b, want_b) and np.array_equal(s, want_s), f"round {rnd}"
        for x, y in zip(b.tolist(), sh.tolist()):   # surviving entries keep their shadow
            if x in shadow_of and live.get(x) is not None and x not in freed:
                assert shadow_of[x] == y
        shadow_of = dict(zip(b.tolist(), sh.tolist()))
        freed = {}
    st = ctx.stats()
    assert st["table_uploads"] == uploads and st["table_merges"] >= 1
    U.assert_same_state(ctx, orc, v, None)


def test_large_table_merge_and_free_all(cg):
    """100,000 allocations, then 3% of them freed and 1,000 registered: one
    merge; then every allocation freed: an empty device table."""
    rng = random.Random(5)
    w = S.small(3)
    ctx, orc, _ = U.make_pair(w.image, None)
    n = 100_000
    bases = np.arange(n, dtype=np.uint64) * np.uint64(1 << 16) + np.uint64(1 << 30)
    sizes = np.array([rng.randrange(1, 1 << 16) for _ in range(n)], dtype=np.uint64)
    assert not ctx.register_allocs(bases, sizes).any()
    live = dict(zip(bases.tolist(), sizes.tolist()))
    b, s, _ = ctx.device_table()
    assert np.array_equal(b, bases) and np.array_equal(s, sizes)
    for x in rng.sample(sorted(live), 3000):
        assert ctx.free(x) == "OK"
        del live[x]
    for k in range(1000):
        x = (1 << 40) + k * (1 << 16)
        assert ctx.register_alloc(x, 4096) == 0
        live[x] = 4096
    b, s, _ = ctx.device_table()
    want_b, want_s = _live_sorted(live)
    assert np.array_equal(b, want_b) and np.array_equal(s, want_s)
    assert ctx.stats()["table_merges"] == 1
    for x in list(live):
        assert ctx.free(x) == "OK"
    b, s, _ = ctx.device_table()
    assert b.size == 0 and ctx.stats()["live_allocs"] == 0
    assert orc is not None

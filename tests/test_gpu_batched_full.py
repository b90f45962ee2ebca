"""The batched workload at full size: 100,000 copies of 16 B-64 MiB against a
1,000,000-entry allocation table, 1 GiB host image, in the launch
configuration the benchmark times (default segment size, TMA engine).

* Carry on, against the oracle: the workload's first 5,000 requests as one
  batch give exactly the oracle's reports and records (the oracle applies
  them one after another in request order), its final host V image, and
  the device shadow of every allocation a copy of the batch wrote.
* Carry off, against the oracle: every copy is then independent, so the
  oracle checks all 100,000 on one shared (read-only) state from several
  threads; every report and record of the whole batch is compared.
* Carry on, the whole batch (device lookup, dependency levels, segmented
  persistent kernels, record compaction) gives exactly the reports, host V
  image and device shadows of the same copies checked one by one with
  cg_check_copy (host lookup, single-copy kernel)."""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import cg_synth as S
import oracle as O
from tests import gpu_util as U

pytestmark = pytest.mark.gpu

PREFIX = 5000


@pytest.fixture(scope="module")
def workload():
    return S.batched(0)


def _ctx(cg, w, carry):
    import torch
    n_img = w.image.n
    a = torch.from_numpy(w.image.a_bits[: n_img // 8].copy()).cuda()
    v = torch.from_numpy(w.image.v.copy()).cuda()
    ctx = cg.Context(carry=carry)
    ctx.bind_host_shadow(a, v)
    order = np.argsort(w.table.base)
    st = ctx.register_allocs(w.table.base[order], w.table.size[order])
    assert not st.any()
    return ctx, v


def _oracle(w, carry):
    orc = O.Oracle(w.image.a_bits, w.image.v, carry=carry)
    order = np.argsort(w.table.base)
    for b, s in zip(w.table.base[order], w.table.size[order]):
        assert orc.register_alloc(int(b), int(s)) == 0
    return orc


def _written_allocations(w, reqs, reps):
    """Indices of the allocations a batch's carries wrote: destinations of
    host->device and device->device copies whose device ranges were valid."""
    bad = O.FLAGS["UNALLOC_DST"] | O.FLAGS["OVERRUN_DST"] | O.FLAGS["UNALLOC_SRC"] | \
        O.FLAGS["OVERRUN_SRC"]
    order = np.argsort(w.table.base)
    sb = w.table.base[order]
    out = set()
    for q, r in zip(reqs, reps):
        if int(q["kind"]) == S.DTOH or r["flags"] & bad or int(q["n"]) == 0:
            continue
        j = int(np.searchsorted(sb, np.uint64(q["dst"]), side="right")) - 1
        out.add(int(order[j]))
    return sorted(out)


def test_batch_prefix_against_oracle_carry(workload):
    import torch

    import paper_1310_0901_gb300 as cg
    w = workload
    reqs = w.reqs[:PREFIX]
    ctx, v = _ctx(cg, w, True)
    st, reps, recs, total, _ = ctx.check_batch(reqs, rec_cap=8 * len(reqs))
    assert st == 0, cg.cg_last_error()
    got = U.reports_from_array(reps)
    assert ctx.stats()["levels"] > 1
    orc = _oracle(w, True)
    st_o, oreps, _ = orc.check_batch(reqs)
    assert st_o == 0
    for i, (g, o) in enumerate(zip(got, oreps)):
        if g != o:
            U.assert_same_report(g, o, f"request {i}")
    orecs = O.emit_records(oreps, reqs)
    assert total == len(orecs)
    assert U.reports_from_array(recs) == orecs
    gv = v.cpu().numpy()
    ov = orc.read_host_v()
    if not np.array_equal(gv, ov):
        bad = np.nonzero(gv != ov)[0]
        raise AssertionError(f"host V differs at {bad[:10]} (of {bad.size})")
    written = _written_allocations(w, reqs, oreps)
    assert len(written) > 100
    for j in written:
        b, s = int(w.table.base[j]), int(w.table.size[j])
        if not np.array_equal(ctx.read_device_shadow(b, s), orc.read_dev_v(b, s)):
            raise AssertionError(f"device shadow of allocation {j} differs")
    orc.close()
    ctx.close()
    del ctx, v
    torch.cuda.empty_cache()


def test_whole_batch_against_oracle_no_carry(workload):
    import torch

    import paper_1310_0901_gb300 as cg
    w = workload
    ctx, v = _ctx(cg, w, False)
    st, reps, recs, total, _ = ctx.check_batch(w.reqs, rec_cap=8 * len(w.reqs))
    assert st == 0
    got = U.reports_from_array(reps)
    recs = U.reports_from_array(recs)
    ctx.close()
    del ctx, v
    torch.cuda.empty_cache()
    # without the carry a check changes no state: one oracle state, read by
    # several threads at once (the oracle is a C library; ctypes calls run
    # without the interpreter lock)
    orc = _oracle(w, False)
    nthreads = max(1, min(16, os.cpu_count() or 1))
    parts = [np.arange(t, len(w.reqs), nthreads) for t in range(nthreads)]

    def run(idx):
        st_o, r, _ = orc.check_batch(w.reqs[idx])
        assert st_o == 0
        return r

    with ThreadPoolExecutor(nthreads) as ex:
        results = list(ex.map(run, parts))
    oreps = [None] * len(w.reqs)
    for idx, r in zip(parts, results):
        for i, o in zip(idx, r):
            oreps[i] = o
    for i, (g, o) in enumerate(zip(got, oreps)):
        if g != o:
            U.assert_same_report(g, o, f"request {i}")
    orecs = O.emit_records(oreps, w.reqs)
    assert total == len(orecs)
    assert recs == orecs
    orc.close()


def test_batch_equals_one_by_one(workload):
    import torch

    import paper_1310_0901_gb300 as cg
    w = workload
    rng = np.random.default_rng(1)
    live = rng.choice(len(w.table.base), 300, replace=False)
    ctx, v = _ctx(cg, w, True)
    st, reps, recs, total, _ = ctx.check_batch(w.reqs, rec_cap=8 * len(w.reqs))
    assert st == 0, cg.cg_last_error()
    batch_reps = U.reports_from_array(reps)
    batch_v = v.cpu().numpy()
    shadows = [ctx.read_device_shadow(int(w.table.base[j]), int(w.table.size[j])) for j in live]
    assert ctx.stats()["levels"] > 1
    ctx.close()
    del ctx, v
    torch.cuda.empty_cache()
    ctx, v = _ctx(cg, w, True)
    for i, q in enumerate(w.reqs):
        st, g = ctx.check_copy(int(q["kind"]), int(q["dst"]), int(q["src"]), int(q["n"]))
        assert st == 0
        if g != batch_reps[i]:
            U.assert_same_report(batch_reps[i], g, f"request {i}")
    assert np.array_equal(v.cpu().numpy(), batch_v)
    for j, sh in zip(live, shadows):
        assert np.array_equal(ctx.read_device_shadow(int(w.table.base[j]), int(w.table.size[j])), sh)
    ctx.close()

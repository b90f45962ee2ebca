"""The batched workload at full size: 100,000 copies of 16 B-64 MiB against a
1,000,000-entry allocation table, 1 GiB host image, in the launch
configuration the benchmark times (default segment size, TMA engine).

* With the carry on, the batch (device lookup, dependency levels,
  segmented persistent kernels, record compaction) gives exactly the
  reports, host V image and device shadow of the same copies checked one by
  one with cg_check_copy (host lookup, single-copy kernel).
* With the carry off every copy is independent, so the oracle can check a
  sample of them one by one, field by field, and the records of the whole
  batch follow from the reports."""
from __future__ import annotations

import numpy as np
import pytest

import cg_synth as S
import oracle as O
from tests import gpu_util as U

pytestmark = pytest.mark.gpu


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


def test_batch_against_oracle_sampled(workload):
    import paper_1310_0901_gb300 as cg
    w = workload
    ctx, v = _ctx(cg, w, False)
    st, reps, recs, total, _ = ctx.check_batch(w.reqs, rec_cap=8 * len(w.reqs))
    assert st == 0
    got = U.reports_from_array(reps)
    orc = O.Oracle(w.image.a_bits, w.image.v, carry=False)
    order = np.argsort(w.table.base)
    for b, s in zip(w.table.base[order], w.table.size[order]):
        assert orc.register_alloc(int(b), int(s)) == 0
    rng = np.random.default_rng(2)
    sample = rng.choice(len(w.reqs), 400, replace=False)
    sample = sample[w.reqs["n"][sample] <= (16 << 20)]  # keep the oracle quick
    for i in sample:
        q = w.reqs[i]
        st_o, o = orc.check_copy(int(q["kind"]), int(q["dst"]), int(q["src"]), int(q["n"]))
        assert st_o == 0
        U.assert_same_report(got[i], o, f"request {i}")
    # records: the oracle's emission rule applied to the batch's own reports
    orecs = O.emit_records(got, w.reqs)
    assert total == len(orecs)
    assert U.reports_from_array(recs) == orecs
    ctx.close()

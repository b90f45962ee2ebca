"""The adversarial error-density workload at its full size: 10,000 copies of
4 KiB-16 MiB (60/30/10 host->device / device->host / device->device) over a
1 GiB host image in which half of the bytes carry random partial V masks and
5 % are unaddressable, against 1,024 allocations of 4 KiB-32 MiB; carry on,
one batch.

Every copy reports.  The batch must give exactly the oracle's reports and
records (the oracle applies the copies one after another in request order),
its final host V image and the device shadow of every allocation."""
from __future__ import annotations

import numpy as np
import pytest

import cg_synth as S
import oracle as O
from tests import gpu_util as U

pytestmark = pytest.mark.gpu


def test_adversarial_full_size_against_oracle():
    import torch

    import paper_1310_0901_gb300 as cg
    w = S.adversarial(0)
    assert len(w.reqs) == 10_000 and w.image.n == 1 << 30
    ctx, orc, (a, v) = U.make_pair(w.image, w.table)
    st, reps, recs, total, _ = ctx.check_batch(w.reqs, rec_cap=8 * len(w.reqs))
    assert st == 0, cg.cg_last_error()
    assert ctx.stats()["levels"] > 1
    got = U.reports_from_array(reps)
    st_o, oreps, _ = orc.check_batch(w.reqs)
    assert st_o == 0
    for i, (g, o) in enumerate(zip(got, oreps)):
        if g != o:
            U.assert_same_report(g, o, f"adversarial request {i}")
    assert all(o["flags"] for o in oreps)  # every copy reports
    orecs = O.emit_records(oreps, w.reqs)
    assert total == len(orecs) and U.reports_from_array(recs) == orecs
    U.assert_same_state(ctx, orc, v, w.table)
    ctx.close()
    orc.close()
    del a, v
    torch.cuda.empty_cache()

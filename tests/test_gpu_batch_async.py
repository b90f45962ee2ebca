"""Asynchronous batches: with two batches in flight (the next one looked up
and planned while the one before runs), every batch's reports, records and
the final shadow state equal those of the same batches checked one after
another with cg_check_batch, and the oracle's."""
from __future__ import annotations

import numpy as np
import pytest

import cg_synth as S
import oracle as O
from tests import gpu_util as U

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cg():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1310_0901_gb300 as m
    return m


@pytest.mark.parametrize("seed,engine,direct", [(0, 0, 0), (1, 1, 0), (2, 0, 1)])
def test_pipelined_batches_equal_sequential(cg, seed, engine, direct):
    """direct = 0: every batch's kernels run as a CUDA graph (updated in place
    for batches of the same shape); 1: launched one by one."""
    w = S.small(seed)
    parts = np.array_split(w.reqs, 6)
    ctx_a, orc, (a_a, v_a) = U.make_pair(w.image, w.table, scan_engine=engine,
                                         batch_direct_launch=direct)
    ctx_b, _, (a_b, v_b) = U.make_pair(w.image, w.table, scan_engine=engine,
                                       batch_direct_launch=1 - direct)
    pending = []
    got = []
    for p in parts:
        st, t, _ = ctx_a.check_batch_async(p)
        assert st == 0, cg.cg_last_error()
        pending.append((t, len(p)))
        if len(pending) == 2:
            t0, n0 = pending.pop(0)
            got.append(ctx_a.batch_wait(t0, n0))
    for t0, n0 in pending:
        got.append(ctx_a.batch_wait(t0, n0))
    for i, (p, (st, reps, recs, total)) in enumerate(zip(parts, got)):
        assert st == 0
        st_b, reps_b, recs_b, total_b, _ = ctx_b.check_batch(p)
        st_o, oreps, _ = orc.check_batch(p)
        assert st_b == st_o == 0
        for j, (g, o) in enumerate(zip(U.reports_from_array(reps), oreps)):
            U.assert_same_report(g, o, f"pipelined batch {i} request {j}")
        assert total == total_b == len(O.emit_records(oreps, p))
        assert U.reports_from_array(recs) == U.reports_from_array(recs_b[:total_b])
    U.assert_same_state(ctx_a, orc, v_a, w.table)
    assert np.array_equal(v_a.cpu().numpy(), v_b.cpu().numpy())


def test_async_batch_limits(cg):
    w = S.small(4)
    ctx, _, _ = U.make_pair(w.image, w.table)
    p = w.reqs[:300]
    st1, t1, _ = ctx.check_batch_async(p)
    st2, t2, _ = ctx.check_batch_async(p)
    assert st1 == st2 == 0 and t1 != t2
    st3, _, _ = ctx.check_batch_async(p)
    assert st3 == -14                                   # two in flight at most
    args = np.zeros(1, S.KARG_DTYPE)
    args[0] = (int(w.table.base[0]), 8, S.ARG_READ, 0)
    assert ctx.check_kernel_args(args)[0] == -12        # slots busy
    assert ctx.batch_wait(t2, len(p))[0] == 0          # out of order is fine
    assert ctx.batch_wait(t1, len(p))[0] == 0
    assert ctx.batch_wait(t1, len(p))[0] == -1          # already collected
    bad = p.copy()
    bad[7]["kind"] = 9
    st, _, idx = ctx.check_batch_async(bad)
    assert st == -2 and idx == 7
    assert ctx.check_kernel_args(args)[0] == 0

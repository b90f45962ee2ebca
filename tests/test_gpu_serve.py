"""Serving: requests from several client threads are admitted in one global
order (result.seq) and their checks are batched into rounds that overlap on
the GPU.  Each result must equal what the same request gets when every
request is applied alone, one by one, in seq order -- on a fresh libcg
context through the single-call API, and in the CPU oracle."""
from __future__ import annotations

import numpy as np
import pytest

import cg_synth as S
import oracle as O
from tests import gpu_util as U

races_found = []

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cg():
    import torch
    assert torch.cuda.is_available()
    import paper_1310_0901_gb300 as m
    return m


def _apply_alone(cg, ctx, orc, q):
    """One request through the single-call API and the oracle; returns
    (status, verdict name or None, report or None), asserting they agree."""
    op, kind, d, s, n = (int(q["op"]), int(q["kind"]), int(q["dst"]), int(q["src"]),
                         int(q["n"]))
    if op == cg.OP_CHECK:
        st, g = ctx.check_copy(kind, d, s, n)
        st_o, o = orc.check_copy(kind, d, s, n)
        assert st == st_o
        if st == 0:
            U.assert_same_report(g, o, f"alone {q}")
        return st, None, g
    if op == cg.OP_ALLOC:
        st = ctx.register_alloc(d, n)
        assert st == orc.register_alloc(d, n)
        return st, None, None
    if op == cg.OP_FREE:
        v = ctx.free(d)
        assert v == orc.free(d)
        return 0, v, None
    val = 0 if op == cg.OP_MARK_DEFINED else 0xFF
    st = ctx.mark_defined(d, n) if op == cg.OP_MARK_DEFINED else ctx.mark_undefined(d, n)
    assert st == orc.mark(d, n, val)
    return st, None, None


@pytest.mark.parametrize("streams,budget,max_round", [(2, 1 << 18, 64), (3, 1 << 30, 512),
                                                     (1, 1 << 16, 16)])
def test_served_results_equal_alone(cg, streams, budget, max_round):
    w = S.small(3)
    rng = S.rng_for(11 + streams)
    live = np.setdiff1d(np.arange(len(w.table.base)), w.table.freed)
    targets = S.AllocTable(w.table.base[live], w.table.size[live], np.zeros(0, np.int64))
    tr = S.serve_trace(rng, 4000, 4e6, 4, targets, w.image.n,
                       size_mix=((0.7, 1, 4096), (0.3, 4096, 16384)), event_frac=0.08,
                       dyn_slots_per_client=48, mark_frac=0.01)
    ctx, _, (a, v) = U.make_pair(w.image, w.table)
    ctx.serve_start(clients=4, ring_capacity=256, max_round=max_round, streams=streams,
                    budget_bytes=budget)
    # while serving, the single-call API is refused
    assert ctx.check_copy(S.HTOD, int(w.table.base[live[0]]), 0, 16)[0] == -12
    res = ctx.serve_replay(tr.reqs, tr.client, tr.arrival_ns)
    stats = ctx.serve_stop()
    n = len(tr.reqs)
    assert sorted(res["seq"].tolist()) == list(range(n))
    assert stats["requests"] == n and stats["rounds"] > 1
    for c in range(4):  # each client's requests take effect in its submission order
        seqs = res["seq"][tr.client == c]
        assert np.all(np.diff(seqs.astype(np.int64)) > 0)
    lat = (res["done_ns"] - res["submit_ns"]).astype(np.int64)
    assert np.all(lat >= 0)
    # replay alone, in seq order, on a fresh context and in the oracle
    ctx2, orc, (a2, v2) = U.make_pair(w.image, w.table)
    names = cg.REPORT_DTYPE.names
    order = np.argsort(res["seq"])
    alone = {}
    for i in order:
        q = tr.reqs[i]
        st, verdict, rep = _apply_alone(cg, ctx2, orc, q)
        assert int(res["status"][i]) == st, (i, q, int(res["status"][i]), st)
        if verdict is not None:
            assert cg.FREE_NAMES[int(res["verdict"][i])] == verdict, (i, q)
        if rep is not None and st == 0:
            alone[i] = rep
    # the concurrent-access class: the oracle's definition over the recorded
    # submit and result times (copies that moved data: valid device ranges)
    dev_fail = sum(O.FLAGS[k] for k in ("UNALLOC_DST", "UNALLOC_SRC", "OVERRUN_DST",
                                        "OVERRUN_SRC"))
    moved = np.array([i in alone and alone[i]["expected"] > 0 and not alone[i]["flags"] & dev_fail
                      for i in order], dtype=np.uint8)
    race = O.races(tr.reqs[order], tr.client[order], res["submit_ns"][order],
                   res["done_ns"][order], moved)
    for k, i in enumerate(order):
        if i not in alone:
            continue
        want = dict(alone[i])
        if race[k] >= 0:
            want["flags"] |= O.FLAGS["CONCURRENT"]
            want["race_seq"] = int(race[k])
        got = {f: int(res["report"][i][f]) for f in names}
        U.assert_same_report(got, want, f"served request {i} (seq {int(res['seq'][i])})")
    races_found.append(int((race >= 0).sum()))
    assert np.array_equal(v.cpu().numpy(), v2.cpu().numpy())
    assert np.array_equal(v.cpu().numpy(), orc.read_host_v())


def test_serving_api_edges(cg):
    w = S.small(4)
    ctx, _, _ = U.make_pair(w.image, w.table)
    ctx.serve_start(clients=2, ring_capacity=4, max_round=8, streams=2)
    st, _ = ctx.submit(5, cg.OP_CHECK, S.HTOD, int(w.table.base[0]), 0, 8)
    assert st == -1  # no such client
    tickets = []
    for k in range(4):
        st, t = ctx.submit(0, cg.OP_CHECK, S.HTOD, int(w.table.base[0]), 0, 8)
        assert st == 0
        tickets.append(t)
    st, _ = ctx.submit(0, cg.OP_CHECK, S.HTOD, int(w.table.base[0]), 0, 8)
    assert st == -14  # ring full until results are collected
    for t in tickets:
        st, r = ctx.wait(t)
        assert st == 0 and r.status == 0 and r.report.expected == 8
    st, r = ctx.wait(tickets[0], 10)
    assert st == -1  # already collected
    st, t = ctx.submit(1, 77, 0, 0, 0, 0)  # unknown op: its own error, served
    assert st == 0
    st, r = ctx.wait(t)
    assert st == 0 and r.status == -1
    ctx.serve_stop()
    assert ctx.check_copy(S.HTOD, int(w.table.base[0]), 0, 8)[0] == 0  # usable again


def test_some_races_were_exercised():
    """The mixes above (4 clients arriving at 4M req/s over a 1 MiB image)
    must have produced concurrent-access findings, or the class went
    untested."""
    if not races_found:
        pytest.skip("serving tests did not run")
    assert sum(races_found) > 0, races_found

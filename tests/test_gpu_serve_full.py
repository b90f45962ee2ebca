"""The serving workload at its full shape, against the oracle: 8 client
streams with Poisson arrivals at 200k requests/s (checks of 1 B-256 MiB,
allocation and free events at 5 % of the traffic), 100,100 allocations and a
32 GiB host image resident in device memory, served with the benchmark's
configuration (4 streams, rounds of up to 8,192 copies, 8 GiB budget).

The trace is the serving generator run for half a second (about 100,000
requests).  Every served result must equal the oracle's for the same request
when the oracle applies all requests one by one in the served order
(result.seq), with the concurrent-access class given by the oracle's own
definition over the recorded submit and result times.  Afterwards the whole
host V image and the device shadow of the allocations the trace wrote (all
small ones, a sample of the 256 MiB ones) must equal the oracle's."""
from __future__ import annotations

import numpy as np
import pytest

import cg_synth as S
import oracle as O
from tests import gpu_util as U

pytestmark = pytest.mark.gpu

SLICE_S = 0.5
HOST_N = 32 << 30


def _image():
    """The serving image (fully addressable, planted undefined runs) on the
    host: V and the packed A bits."""
    vh = np.zeros(HOST_N, np.uint8)
    starts, lengths, values = S.serving_image_runs(0, HOST_N)
    for s0, ln, val in zip(starts, lengths, values):
        vh[s0:s0 + ln] = val
    idx = np.unique(np.concatenate([np.arange(s0, s0 + ln) for s0, ln in zip(starts, lengths)]))
    return vh, idx


def test_serving_slice_against_oracle():
    import torch

    import paper_1310_0901_gb300 as cg
    tr = S.serving(0, seconds=SLICE_S, host_n=HOST_N)
    vh, idx = _image()
    dev = torch.device("cuda", 0)
    v = torch.zeros(HOST_N, dtype=torch.uint8, device=dev)
    a = torch.full((HOST_N // 8,), 0xFF, dtype=torch.uint8, device=dev)
    v[torch.from_numpy(idx).to(dev)] = torch.from_numpy(vh[idx]).to(dev)
    ctx = cg.Context()
    ctx.bind_host_shadow(a, v)
    order = np.argsort(tr.table.base)
    assert not ctx.register_allocs(tr.table.base[order], tr.table.size[order]).any()
    ctx.serve_start(clients=8, ring_capacity=1 << 14, max_round=8192, streams=4,
                    budget_bytes=8 << 30)
    res = ctx.serve_replay(tr.reqs, tr.client, tr.arrival_ns)
    stats = ctx.serve_stop()
    n = len(tr.reqs)
    assert stats["requests"] == n and stats["rounds"] > 1
    assert sorted(res["seq"].tolist()) == list(range(n))

    orc = O.Oracle(np.full(HOST_N // 8, 0xFF, np.uint8), vh)
    del vh
    for b, s in zip(tr.table.base[order], tr.table.size[order]):
        assert orc.register_alloc(int(b), int(s)) == 0
    names = cg.REPORT_DTYPE.names
    seq_order = np.argsort(res["seq"])
    alone = {}
    written = set()  # bases of live allocations a copy wrote
    live_size = dict(zip(tr.table.base.tolist(), tr.table.size.tolist()))
    dev_fail = sum(O.FLAGS[k] for k in ("UNALLOC_DST", "UNALLOC_SRC", "OVERRUN_DST",
                                        "OVERRUN_SRC"))
    for i in seq_order:
        q = tr.reqs[i]
        op, kind, d, s, m = (int(q["op"]), int(q["kind"]), int(q["dst"]), int(q["src"]),
                             int(q["n"]))
        if op == cg.OP_CHECK:
            st, o = orc.check_copy(kind, d, s, m)
            assert int(res["status"][i]) == st, (i, q)
            if st == 0:
                alone[i] = o
                if kind != S.DTOH and m and not o["flags"] & dev_fail:
                    written.add(int(o["alloc_base_dst"]))
        elif op == cg.OP_ALLOC:
            st = orc.register_alloc(d, m)
            assert int(res["status"][i]) == st, (i, q)
            if st == 0:
                live_size[d] = m
        elif op == cg.OP_FREE:
            verdict = orc.free(d)
            assert cg.FREE_NAMES[int(res["verdict"][i])] == verdict, (i, q)
            if verdict == "OK":
                live_size.pop(d)
                written.discard(d)
        else:
            st = orc.mark(d, m, 0 if op == cg.OP_MARK_DEFINED else 0xFF)
            assert int(res["status"][i]) == st, (i, q)
    # the concurrent-access class over the recorded times (copies that moved
    # data: valid device ranges)
    moved = np.array([i in alone and alone[i]["expected"] > 0 and
                      not alone[i]["flags"] & dev_fail for i in seq_order], dtype=np.uint8)
    race = O.races(tr.reqs[seq_order], tr.client[seq_order], res["submit_ns"][seq_order],
                   res["done_ns"][seq_order], moved)
    n_checked = 0
    for k, i in enumerate(seq_order):
        if i not in alone:
            continue
        want = dict(alone[i])
        if race[k] >= 0:
            want["flags"] |= O.FLAGS["CONCURRENT"]
            want["race_seq"] = int(race[k])
        got = {f: int(res["report"][i][f]) for f in names}
        if got != want:
            U.assert_same_report(got, want, f"served request {i} (seq {int(res['seq'][i])})")
        n_checked += 1
    assert n_checked > 0.9 * n
    # final state: the whole host V image, in 1 GiB pieces
    piece = 1 << 30
    for off in range(0, HOST_N, piece):
        g = v[off:off + piece].cpu().numpy()
        o = orc.read_host_v(off, piece)
        if not np.array_equal(g, o):
            bad = np.nonzero(g != o)[0]
            raise AssertionError(f"host V differs at {off + bad[:10]}")
    # device shadows the trace wrote: every small allocation, ten 256 MiB ones
    sizes = live_size
    big = sorted(b for b in written if sizes[b] >= (256 << 20))
    small = sorted(b for b in written if sizes[b] < (256 << 20))
    rng = np.random.default_rng(5)
    sample = small + [big[j] for j in rng.permutation(len(big))[:10]]
    assert len(small) > 1000 and big
    for b in sample:
        if not np.array_equal(ctx.read_device_shadow(b, sizes[b]), orc.read_dev_v(b, sizes[b])):
            raise AssertionError(f"device shadow of the allocation at {b:#x} differs")
    orc.close()
    ctx.close()
    del a, v
    torch.cuda.empty_cache()

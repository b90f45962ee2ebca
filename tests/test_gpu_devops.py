"""GPU parity of the memset wrappers' check and of kernel-argument checks
against the CPU oracle, bit-exact.

Memsets, kernel launches and ordinary copies are interleaved on one context
and one oracle state (so definedness flows between them: copies define
device bytes, reads of arguments count what is still undefined, write
arguments and memsets define their ranges); every status, report and the
final shadow state must be equal.  The full-size case is the benchmark's:
a 1 GiB memset and one launch with four 256 MiB arguments."""
from __future__ import annotations

import collections

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


def _karg_reports(cg, reps):
    return U.reports_from_array(reps)


@pytest.mark.parametrize("seed,carry,engine,strict", [(0, True, 0, False), (1, True, 1, False),
                                                      (2, False, 0, False), (3, True, 0, True)])
def test_interleaved_memsets_launches_copies(cg, seed, carry, engine, strict):
    w = S.small(seed)
    ctx, orc, (a, v) = U.make_pair(w.image, w.table, carry=carry, strict=strict,
                                   scan_engine=engine)
    rng = S.rng_for(100 + seed)
    launches = S.kernel_launches(rng, 150, w.table, bytes_hi=16 << 10)
    sets = S.memsets(rng, 150, w.table)
    seen = collections.Counter()
    for step in range(300):
        u = rng.random()
        if u < 0.35:
            q = w.reqs[int(rng.integers(0, len(w.reqs)))]
            k, d, s_, n = int(q["kind"]), int(q["dst"]), int(q["src"]), int(q["n"])
            st_g, g = ctx.check_copy(k, d, s_, n)
            st_o, o = orc.check_copy(k, d, s_, n)
            assert st_g == st_o
            if st_o == 0:
                U.assert_same_report(g, o, f"copy at step {step}")
        elif u < 0.65:
            d, pitch, wd, h = sets.pop()
            st_g, g = ctx.check_memset(d, wd, h, pitch)
            st_o, o = orc.memset(d, wd, h, pitch)
            assert st_g == st_o, (step, st_g, st_o)
            if st_o == 0:
                U.assert_same_report(g, o, f"memset at step {step}")
                seen["memset_bad" if o["flags"] else "memset_ok"] += 1
        else:
            args = launches.pop()
            st_g, reps, _ = ctx.check_kernel_args(args)
            st_o, oreps = orc.check_kernel_args(args["ptr"], args["bytes"], args["access"])
            assert st_g == st_o == 0, (step, cg.cg_last_error())
            for i, (g, o) in enumerate(zip(U.reports_from_array(reps), oreps)):
                U.assert_same_report(g, o, f"launch at step {step}, argument {i}")
                for name, bit in O.FLAGS.items():
                    if o["flags"] & bit:
                        seen[name] += 1
        if step % 60 == 59:
            U.assert_same_state(ctx, orc, v, w.table)
    U.assert_same_state(ctx, orc, v, w.table)
    for k in ("memset_ok", "memset_bad", "DEV_UNDEF_SRC", "OVERRUN_SRC", "OVERRUN_DST"):
        assert seen[k] > 0, (k, seen)


def test_kernel_arg_edges(cg):
    """Refused calls change nothing and name the argument; an empty launch;
    zero extents (pointer containment only); an argument read and written
    in the same launch reports what was undefined before it; interior and
    freed pointers."""
    w = S.small(7)
    ctx, orc, (a, v) = U.make_pair(w.image, w.table)
    live = np.setdiff1d(np.arange(len(w.table.base)), w.table.freed)
    b0, s0 = int(w.table.base[live[0]]), int(w.table.size[live[0]])
    fb = int(w.table.base[w.table.freed[0]])
    R, W = S.ARG_READ, S.ARG_WRITE
    bad = np.array([(b0, 10, R, 0), (b0, 10, 4, 0)], S.KARG_DTYPE)
    st, _, idx = ctx.check_kernel_args(bad)
    assert st == -1 and idx == 1
    bad = np.array([(b0, 10, 0, 0)], S.KARG_DTYPE)
    assert ctx.check_kernel_args(bad)[0] == -1
    bad = np.array([(b0, 10, R, 7)], S.KARG_DTYPE)
    assert ctx.check_kernel_args(bad)[0] == -1
    st, reps, _ = ctx.check_kernel_args(np.zeros(0, S.KARG_DTYPE))
    assert st == 0 and len(reps) == 0
    cases = np.array([
        (b0 + 5, 0, R, 0), (b0 + s0, 0, R | W, 0), (fb, 0, W, 0), (b0, s0, R | W, 0),
        (b0, s0, R, 0), (b0 + 3, s0, R, 0), (fb + 1, 8, R, 0), (b0 + 100, 64, W, 0),
    ], S.KARG_DTYPE)
    st, reps, _ = ctx.check_kernel_args(cases)
    st_o, oreps = orc.check_kernel_args(cases["ptr"], cases["bytes"], cases["access"])
    assert st == st_o == 0
    for i, (g, o) in enumerate(zip(U.reports_from_array(reps), oreps)):
        U.assert_same_report(g, o, f"edge argument {i}")
    assert oreps[4]["n_undef"] == s0 == oreps[3]["n_undef"]  # fresh: all undefined, read before
    st, reps, _ = ctx.check_kernel_args(cases[4:5])                # ... the launch defined it
    assert st == 0 and int(reps[0]["n_undef"]) == 0
    assert orc.check_kernel_args(cases["ptr"][4:5], cases["bytes"][4:5],
                                 cases["access"][4:5])[1][0]["n_undef"] == 0
    U.assert_same_state(ctx, orc, v, w.table)


def test_memset_async(cg):
    """cg_check_memset_async writes the report into device memory."""
    import torch
    w = S.small(8)
    ctx, orc, (a, v) = U.make_pair(w.image, w.table)
    rng = S.rng_for(9)
    sets = S.memsets(rng, 40, w.table) + [(12345, 0, 0, 3)]
    reps = torch.zeros((len(sets), cg.REPORT_DTYPE.itemsize), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    want = []
    for i, (d, pitch, wd, h) in enumerate(sets):
        assert cg.cg_check_memset_async(ctx.handle, d, pitch, wd, h, reps[i].data_ptr(), stream) == 0
        want.append(orc.memset(d, wd, h, pitch))
    torch.cuda.synchronize()
    got = np.frombuffer(reps.cpu().numpy().tobytes(), dtype=cg.REPORT_DTYPE)
    for i, (st, o) in enumerate(want):
        assert st == 0
        assert {k: int(got[i][k]) for k in got.dtype.names} == o, i
    U.assert_same_state(ctx, orc, v, w.table)


def test_devops_full_size(cg):
    """The benchmark's workload: a 1 GiB memset, then one launch reading two
    256 MiB buffers (one carrying planted undefined runs), reading and
    writing a third and writing a fourth; against the oracle in full."""
    wl = S.devops_large()
    ctx, orc, (a, v) = U.make_pair(wl.image, wl.table)
    for q in wl.setup:  # host->device copies that define the read buffers
        st_g, g = ctx.check_copy(*q)
        st_o, o = orc.check_copy(*q)
        assert st_g == st_o == 0
        U.assert_same_report(g, o, "setup copy")
    d, pitch, wd, h = wl.memset
    st_g, g = ctx.check_memset(d, wd, h, pitch)
    st_o, o = orc.memset(d, wd, h, pitch)
    assert st_g == st_o == 0 and o["flags"] == 0
    U.assert_same_report(g, o, "1 GiB memset")
    st, reps, _ = ctx.check_kernel_args(wl.args)
    st_o, oreps = orc.check_kernel_args(wl.args["ptr"], wl.args["bytes"], wl.args["access"])
    assert st == st_o == 0
    for i, (g, o) in enumerate(zip(U.reports_from_array(reps), oreps)):
        U.assert_same_report(g, o, f"large argument {i}")
    assert oreps[0]["n_undef"] > 0   # the planted runs are found
    U.assert_same_state(ctx, orc, v, wl.table)

"""Failure paths, exercised without faulting the GPU.

A stalled bulk copy is made on purpose (the injected fault issues no copy
for one tile, so its bounded wait runs out after about a second): the check
must come back flagged incomplete with CG_E_TIMEOUT, within a few seconds,
and the context must stay usable and agree with the oracle afterwards.  An
injected shadow-allocation failure must leave the table unchanged."""
from __future__ import annotations

import ctypes
import time

import numpy as np
import pytest

import cg_synth as S
from tests import gpu_util as U

pytestmark = pytest.mark.gpu

INCOMPLETE = 1 << 31


@pytest.fixture(scope="module")
def cg():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1310_0901_gb300 as m
    return m


def _pair():
    n = 16 << 20
    img = S.host_image_runs(S.rng_for(61), n, undef_frac=1e-4, unaddr_p=1e-5)
    base = 1 << 40
    table = S.AllocTable(np.array([base, base + (64 << 20)], np.uint64),
                         np.array([n, 4096], np.uint64), np.zeros(0, np.int64))
    ctx, orc, (a, v) = U.make_pair(img, table, scan_engine=2)
    return ctx, orc, v, table, base, n


def test_stalled_copy_times_out_then_context_recovers(cg):
    ctx, orc, v, table, base, n = _pair()
    assert cg.cg_inject_fault(ctx.handle, cg.FAULT_STALL_COPY) == 0
    t0 = time.perf_counter()
    st, rep = ctx.check_copy(S.HTOD, base, 0, n)
    elapsed = time.perf_counter() - t0
    assert st == -13, (st, cg.cg_last_error())
    assert "bounded wait" in cg.cg_last_error().decode()
    assert rep["flags"] & INCOMPLETE
    assert 0.5 < elapsed < 30, elapsed
    # the fault was one-shot: the same copy again (its carry rewrites every
    # byte the stalled one wrote) equals the oracle's single application
    st, g = ctx.check_copy(S.HTOD, base, 0, n)
    st_o, o = orc.check_copy(S.HTOD, base, 0, n)
    assert st == st_o == 0
    U.assert_same_report(g, o, "after the stall")
    U.assert_same_state(ctx, orc, v, table)


def test_stalled_async_check_flags_its_report(cg):
    import torch
    ctx, orc, v, table, base, n = _pair()
    rep = torch.zeros(cg.REPORT_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    assert cg.cg_inject_fault(ctx.handle, cg.FAULT_STALL_COPY) == 0
    q = cg.cg_copy(S.HTOD, 0, base, 0, n)
    assert cg.cg_check_copy_async(ctx.handle, ctypes.byref(q), rep.data_ptr(),
                                  torch.cuda.current_stream().cuda_stream) == 0
    torch.cuda.synchronize()
    r = np.frombuffer(rep.cpu().numpy().tobytes(), dtype=cg.REPORT_DTYPE)[0]
    assert int(r["flags"]) & INCOMPLETE
    # the next launch starts from a clean scratch area
    assert cg.cg_check_copy_async(ctx.handle, ctypes.byref(q), rep.data_ptr(),
                                  torch.cuda.current_stream().cuda_stream) == 0
    torch.cuda.synchronize()
    r = np.frombuffer(rep.cpu().numpy().tobytes(), dtype=cg.REPORT_DTYPE)[0]
    st_o, o = orc.check_copy(S.HTOD, base, 0, n)
    assert {k: int(r[k]) for k in r.dtype.names} == o


def test_injected_shadow_alloc_failure(cg):
    ctx, orc, v, table, base, n = _pair()
    live = ctx.stats()["live_allocs"]
    assert cg.cg_inject_fault(ctx.handle, cg.FAULT_SHADOW_ALLOC) == 0
    assert ctx.register_alloc(1 << 44, 4096) == -7
    assert "injected" in cg.cg_last_error().decode()
    assert ctx.stats()["live_allocs"] == live
    assert ctx.check_copy(S.HTOD, 1 << 44, 0, 16)[1]["flags"] & 1  # still unallocated
    assert ctx.register_alloc(1 << 44, 4096) == 0                 # one-shot
    assert cg.cg_inject_fault(ctx.handle, cg.FAULT_SHADOW_ALLOC) == 0
    assert ctx.register_array(0x77, 64, 4) == -7
    assert ctx.register_array(0x77, 64, 4) == 0
    assert cg.cg_inject_fault(ctx.handle, 8) == -1

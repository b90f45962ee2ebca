"""Checkpoint / resume: a context saved half-way through a workload and
restored into a fresh context gives, for the second half, the same reports
and the same final shadow state as the context that kept running, and as
the oracle.  Freed bases (double frees) and arrays survive the round trip;
bad files and non-empty targets are refused."""
from __future__ import annotations

import os

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


def test_snapshot_restore_continues_identically(cg, tmp_path):
    import torch
    w = S.small(5)
    ctx, orc, (a, v) = U.make_pair(w.image, w.table)
    for h, W, H, D in [(0x900, 64, 8, 2), (0x901, 32, 4, 1)]:
        assert ctx.register_array(h, W, H, D) == orc.register_array(h, W, H, D) == 0
    half = len(w.reqs) // 2
    for q in w.reqs[:half]:
        args = (int(q["kind"]), int(q["dst"]), int(q["src"]), int(q["n"]))
        st_g, g = ctx.check_copy(*args)
        st_o, o = orc.check_copy(*args)
        assert st_g == st_o
    q3 = dict(kind=S.HTOD, dst=S.side3d(0x900, 0, 0, 3, 1, 1, array=True), src=S.side3d(100, 40),
              width=40, height=5, depth=1)
    assert ctx.check_copy3d(q3["kind"], q3["dst"], q3["src"], 40, 5)[0] == 0
    assert orc.check_copy3d(q3["kind"], q3["dst"], q3["src"], 40, 5)[0] == 0
    assert ctx.free_array(0x901) == orc.free_array(0x901) == "OK"
    path = str(tmp_path / "ctx.cgsnap")
    assert ctx.snapshot(path) == 0, cg.cg_last_error()
    assert os.path.getsize(path) > 8
    # the restored context works on its own copy of the host image
    a2, v2 = a.clone(), v.clone()
    ctx2 = cg.Context()
    ctx2.bind_host_shadow(a2, v2)
    assert ctx2.restore(path) == 0, cg.cg_last_error()
    assert ctx2.stats()["live_allocs"] == ctx.stats()["live_allocs"]
    for q in w.reqs[half:]:
        args = (int(q["kind"]), int(q["dst"]), int(q["src"]), int(q["n"]))
        st1, g1 = ctx.check_copy(*args)
        st2, g2 = ctx2.check_copy(*args)
        st_o, o = orc.check_copy(*args)
        assert st1 == st2 == st_o
        if st_o == 0:
            U.assert_same_report(g2, o, f"restored context, request {args}")
            assert g1 == g2
    torch.cuda.synchronize()
    U.assert_same_state(ctx2, orc, v2, w.table)
    assert np.array_equal(v.cpu().numpy(), v2.cpu().numpy())
    assert np.array_equal(ctx2.read_array_shadow(0x900, 0, 64 * 8 * 2),
                          orc.read_array_v(0x900, 0, 64 * 8 * 2))
    # freed bases and destroyed arrays came along
    fb = int(w.table.base[w.table.freed[0]])
    assert ctx2.free(fb) == "DOUBLE"
    assert ctx2.free_array(0x901) == "DOUBLE"


def test_restore_refusals(cg, tmp_path):
    w = S.small(6)
    ctx, _, _ = U.make_pair(w.image, w.table)
    path = str(tmp_path / "a.cgsnap")
    assert ctx.snapshot(path) == 0
    assert ctx.restore(path) == -12          # not an empty context
    bad = tmp_path / "bad.cgsnap"
    bad.write_bytes(b"NOTASNAP" + b"\0" * 64)
    fresh = cg.Context()
    assert fresh.restore(str(bad)) == -1
    cut = tmp_path / "cut.cgsnap"
    cut.write_bytes(open(path, "rb").read()[:100])
    fresh2 = cg.Context()
    assert fresh2.restore(str(cut)) == -1
    assert "truncated" in cg.cg_last_error().decode()
    assert cg.Context().restore(str(tmp_path / "missing")) == -1

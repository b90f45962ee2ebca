"""Full-size large transfers (256 MiB, 1 GiB, 4 GiB host->device checks with
carry) in the launch configuration the benchmark times.

Each transfer is compared with the oracle field by field, and its whole
carried device shadow byte by byte (read back in 256 MiB pieces).  The
counts and first offset are also checked against what the generator
planted, and the carried shadow against the host V bytes (a fully
addressable source arrives unchanged)."""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

import cg_synth as S
import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def large():
    import torch

    import paper_1310_0901_gb300 as cg
    w = S.large(0)
    n_img = w.image.n
    a = torch.from_numpy(w.image.a_bits[: n_img // 8].copy()).cuda()
    v = torch.from_numpy(w.image.v).cuda()
    ctx = cg.Context()
    ctx.bind_host_shadow(a, v)
    order = np.argsort(w.table.base)
    for b, s in zip(w.table.base[order], w.table.size[order]):
        assert ctx.register_alloc(int(b), int(s)) == 0
    # one oracle over the whole image and table; each transfer writes its
    # own allocation, so the order of the tests does not matter
    orc = O.Oracle(w.image.a_bits, w.image.v)
    for b, s in zip(w.table.base[order], w.table.size[order]):
        assert orc.register_alloc(int(b), int(s)) == 0
    yield cg, ctx, w, (a, v), orc
    orc.close()
    ctx.close()


def _planted(w, n):
    undef = np.zeros(n, bool)
    for s0, ln in w.image.undef_runs:
        if s0 < n:
            undef[s0:min(n, s0 + ln)] = True
    return undef


@pytest.mark.parametrize("idx", [0, 1, 2])
def test_large_transfer(large, idx):
    import torch
    cg, ctx, w, (a, v), orc = large
    q = w.reqs[idx]
    n, dst = int(q["n"]), int(q["dst"])
    # the benchmark's call: asynchronous check, report in device memory
    rep = torch.zeros(cg.REPORT_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    req = cg.cg_copy(int(q["kind"]), 0, dst, int(q["src"]), n)
    st = cg.cg_check_copy_async(ctx.handle, ctypes.byref(req), rep.data_ptr(),
                                torch.cuda.current_stream().cuda_stream)
    assert st == 0
    torch.cuda.synchronize()
    r = np.frombuffer(rep.cpu().numpy().tobytes(), dtype=cg.REPORT_DTYPE)[0]
    undef = _planted(w, n)
    assert int(r["n_undef"]) == int(undef.sum())
    assert int(r["n_unaddr"]) == 0
    assert int(r["n_good"]) == n - int(undef.sum())
    first = int(np.argmax(undef)) if undef.any() else -1
    assert int(r["first_undef_off"]) == first == int(r["first_bad_off"])
    assert int(r["flags"]) == (cg.FLAGS["HOST_UNDEF"] if undef.any() else 0)
    assert int(r["found_dst"]) == int(w.table.size[idx]) and int(r["expected"]) == n
    # carried shadow == host V (fully addressable source), sampled
    rng = np.random.default_rng(idx)
    windows = [(s0 - 64, ln + 128) for s0, ln in w.image.undef_runs if s0 + ln < n][:200]
    windows += [(int(x), 4096) for x in rng.integers(0, n - 4096, 200)]
    windows += [(0, 4096), (n - 4096, 4096)]
    for off, ln in windows:
        off = max(0, off)
        ln = min(ln, n - off)
        got = ctx.read_device_shadow(dst + off, ln)
        assert np.array_equal(got, w.image.v[off:off + ln]), (idx, off)
    # the whole transfer against the oracle: report and carried shadow
    st, o = orc.check_copy(int(q["kind"]), dst, int(q["src"]), n)
    assert st == 0
    assert {k: int(r[k]) for k in r.dtype.names} == o
    piece = 256 << 20
    for off in range(0, n, piece):
        ln = min(piece, n - off)
        got = ctx.read_device_shadow(dst + off, ln)
        want = orc.read_dev_v(dst + off, ln)
        if not np.array_equal(got, want):
            bad = np.nonzero(got != want)[0]
            raise AssertionError(f"transfer {idx}: shadow differs at {off + bad[:10]}")

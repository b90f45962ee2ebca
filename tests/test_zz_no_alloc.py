"""cg_scan_noalloc, the entry point for callers that must not allocate device
memory (for example a checker running inside a wrapped allocation or copy
call, which would re-enter the allocator it wraps), gives the same results
as the ordinary context path cg_check_copy.

Three calls in a row through the C ABI (host->device with carry, an
overlapping device->device carry staged through the library's fixed
scratch array, device->host with carry): each report and the shadow bytes
it leaves behind must equal those of cg_check_copy on the same input.
The file is named to be collected last."""
from __future__ import annotations

import numpy as np
import pytest

import cg_synth as S

pytestmark = pytest.mark.gpu

SCAN_FIELDS = ["flags", "first_bad_kind", "first_bad_off", "first_unaddr_off",
               "first_undef_off", "n_good", "n_unaddr", "n_undef", "expected"]


def _image(n_img, seed):
    rng = np.random.default_rng(seed)
    v = rng.integers(0, 256, n_img).astype(np.uint8)
    v[rng.random(n_img) < 0.7] = 0
    addr = rng.random(n_img) > 0.05
    return S.HostImage(S.pack_a(addr), v, [], None)


def test_noalloc_matches_check_copy():
    import torch

    import paper_1310_0901_gb300 as cg
    from tests import gpu_util as U

    n_img = 1 << 20
    img = _image(n_img, 21)
    base, size = 1 << 36, 1 << 18
    table = S.AllocTable(np.array([base], np.uint64), np.array([size], np.uint64),
                         np.zeros(0, np.int64))
    ctx, _, (_, v_ctx) = U.make_pair(img, table)
    # the allocation-free path works on the caller's own buffers
    a_na = torch.from_numpy(img.a_bits[: n_img // 8].copy()).cuda()
    v_na = torch.from_numpy(img.v.copy()).cuda()
    shadow = torch.full((size,), 0xFF, dtype=torch.uint8, device="cuda")  # a fresh allocation
    reps = torch.zeros((3, cg.REPORT_DTYPE.itemsize), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    sp = shadow.data_ptr()

    calls = [  # (kind, host_off, src shadow offset, dst shadow offset, n)
        (cg.HTOD, 12345, None, 777, 100_000),
        (cg.DTOD, None, 787, 777 + 5000, 60_000),   # source and destination overlap
        (cg.DTOH, 300_001, 1000, None, 90_000),
    ]
    for i, (kind, h, so, do, n) in enumerate(calls):
        if kind == cg.HTOD:
            st, want = ctx.check_copy(kind, base + do, h, n)
        elif kind == cg.DTOD:
            st, want = ctx.check_copy(kind, base + do, base + so, n)
        else:
            st, want = ctx.check_copy(kind, h, base + so, n)
        assert st == 0
        st = cg.cg_scan_noalloc(kind, a_na.data_ptr(), v_na.data_ptr(), n_img,
                                h if h is not None else 0,
                                sp + so if so is not None else None,
                                sp + do if do is not None else None,
                                n, 1, reps[i].data_ptr(), stream)
        assert st == 0, cg.cg_last_error()
        torch.cuda.synchronize()
        got = np.frombuffer(reps[i].cpu().numpy().tobytes(), dtype=cg.REPORT_DTYPE)[0]
        for f in SCAN_FIELDS:
            assert int(got[f]) == int(want[f]), (i, f, int(got[f]), int(want[f]))
        assert want["n_unaddr"] + want["n_undef"] > 0  # the inputs exercise both classes
        assert np.array_equal(shadow.cpu().numpy(), ctx.read_device_shadow(base, size)), i
        assert np.array_equal(v_na.cpu().numpy(), v_ctx.cpu().numpy()), i

    # an overlapping device->device carry beyond the fixed staging area is
    # refused before anything runs
    big = torch.full((20 << 20,), 0x5A, dtype=torch.uint8, device="cuda")
    before = big.clone()
    st = cg.cg_scan_noalloc(cg.DTOD, None, None, 0, 0, big.data_ptr(), big.data_ptr() + 16,
                            (8 << 20) + 16, 1, reps[0].data_ptr(), stream)
    assert st == -15 and "8 MiB" in cg.cg_last_error().decode()
    torch.cuda.synchronize()
    assert torch.equal(big, before)

"""cg_scan_noalloc, the entry point for callers that must not allocate device
memory (for example a checker running inside a wrapped allocation or copy
call, which would re-enter the allocator it wraps), gives the same results
as the CPU oracle and as the ordinary context path cg_check_copy.

One pass is five calls through the C ABI: host->device with carry, an
overlapping device->device carry staged through the library's fixed
scratch array, device->host with carry, a zero-length copy, and a
device->device check with no device shadows (nothing read or carried).
Each report and the shadow bytes it leaves behind must equal the oracle's
(and cg_check_copy's) on the same input.  The pass runs twice in a row; the
second pass must leave the device's free memory unchanged (the first may
load the kernels).  The file is named to be collected last."""
from __future__ import annotations

import numpy as np
import pytest

import cg_synth as S

pytestmark = pytest.mark.gpu

SCAN_FIELDS = ["first_bad_kind", "first_bad_off", "first_unaddr_off",
               "first_undef_off", "n_good", "n_unaddr", "n_undef", "expected"]


def _image(n_img, seed):
    rng = np.random.default_rng(seed)
    v = rng.integers(0, 256, n_img).astype(np.uint8)
    v[rng.random(n_img) < 0.7] = 0
    addr = rng.random(n_img) > 0.05
    return S.HostImage(S.pack_a(addr), v, [], None)


def test_noalloc_matches_oracle_and_check_copy():
    import torch

    import paper_1310_0901_gb300 as cg
    from tests import gpu_util as U

    n_img = 1 << 20
    img = _image(n_img, 21)
    base, size = 1 << 36, 1 << 18
    table = S.AllocTable(np.array([base], np.uint64), np.array([size], np.uint64),
                         np.zeros(0, np.int64))
    ctx, orc, (_, v_ctx) = U.make_pair(img, table)
    # the allocation-free path works on the caller's own buffers
    a_na = torch.from_numpy(img.a_bits[: n_img // 8].copy()).cuda()
    v_na = torch.from_numpy(img.v.copy()).cuda()
    shadow = torch.full((size,), 0xFF, dtype=torch.uint8, device="cuda")  # a fresh allocation
    reps = torch.zeros((5, cg.REPORT_DTYPE.itemsize), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    sp = shadow.data_ptr()
    scan_flags = (cg.FLAGS["HOST_UNADDR"] | cg.FLAGS["HOST_UNDEF"] | cg.FLAGS["DEV_UNDEF_SRC"]
                  | cg.FLAGS["DTOD_OVERLAP"])
    wild_src, wild_dst = 1 << 20, 1 << 24  # outside every allocation: nothing read or carried

    calls = [  # (kind, host_off, src shadow offset, dst shadow offset, n)
        (cg.HTOD, 12345, None, 777, 100_000),
        (cg.DTOD, None, 787, 777 + 5000, 60_000),   # source and destination overlap
        (cg.DTOH, 300_001, 1000, None, 90_000),
        (cg.HTOD, 4096, None, 64, 0),               # zero length: an empty report
        (cg.DTOD, None, None, None, 5000),          # no device shadows
    ]
    free_after = []
    for rnd in range(2):
        for i, (kind, h, so, do, n) in enumerate(calls):
            d_addr = base + do if do is not None else (wild_dst if kind == cg.DTOD else None)
            s_addr = base + so if so is not None else (wild_src if kind == cg.DTOD else None)
            if kind == cg.HTOD:
                args = (kind, d_addr, h, n)
            elif kind == cg.DTOD:
                args = (kind, d_addr, s_addr, n)
            else:
                args = (kind, h, s_addr, n)
            st, want = ctx.check_copy(*args)
            st_o, want_o = orc.check_copy(*args)
            assert st == st_o == 0
            st = cg.cg_scan_noalloc(kind, a_na.data_ptr(), v_na.data_ptr(), n_img,
                                    h if h is not None else 0,
                                    sp + so if so is not None else None,
                                    sp + do if do is not None else None,
                                    n, 1, reps[i].data_ptr(), stream)
            assert st == 0, cg.cg_last_error()
            torch.cuda.synchronize()
            got = np.frombuffer(reps[i].cpu().numpy().tobytes(), dtype=cg.REPORT_DTYPE)[0]
            for f in SCAN_FIELDS:
                assert int(got[f]) == want_o[f] == int(want[f]), (rnd, i, f, int(got[f]), want_o[f])
            assert int(got["flags"]) == want_o["flags"] & scan_flags, (rnd, i)
            if i < 3:  # the inputs exercise both classes
                assert want_o["n_unaddr"] + want_o["n_undef"] > 0
            assert np.array_equal(shadow.cpu().numpy(), orc.read_dev_v(base, size)), (rnd, i)
            assert np.array_equal(shadow.cpu().numpy(), ctx.read_device_shadow(base, size))
            assert np.array_equal(v_na.cpu().numpy(), orc.read_host_v()), (rnd, i)
            assert np.array_equal(v_na.cpu().numpy(), v_ctx.cpu().numpy())
        torch.cuda.synchronize()
        free_after.append(torch.cuda.mem_get_info()[0])
    # the second pass allocated nothing (the first loaded the kernels)
    assert free_after[1] == free_after[0], free_after

    # an overlapping device->device carry beyond the fixed staging area is
    # refused before anything runs
    big = torch.full((20 << 20,), 0x5A, dtype=torch.uint8, device="cuda")
    before = big.clone()
    st = cg.cg_scan_noalloc(cg.DTOD, None, None, 0, 0, big.data_ptr(), big.data_ptr() + 16,
                            (8 << 20) + 16, 1, reps[0].data_ptr(), stream)
    assert st == -15 and "8 MiB" in cg.cg_last_error().decode()
    torch.cuda.synchronize()
    assert torch.equal(big, before)
    # a device shadow in host memory is refused (the bulk copies read device
    # memory only)
    pinned = torch.zeros(4096, dtype=torch.uint8, pin_memory=True)
    st = cg.cg_scan_noalloc(cg.HTOD, a_na.data_ptr(), v_na.data_ptr(), n_img, 0, None,
                            pinned.data_ptr(), 1024, 1, reps[0].data_ptr(), stream)
    assert st == -1 and "device memory" in cg.cg_last_error().decode()
    assert not pinned.any()

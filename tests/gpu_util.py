"""Helpers for the GPU parity tests: one libcg context and one oracle state
fed the same seeded inputs, and exact comparisons between them."""
from __future__ import annotations

import numpy as np

import cg_synth as S
import oracle as O


def torch_cuda():
    import torch
    return torch


def image_tensors(image: S.HostImage):
    torch = torch_cuda()
    n = image.n
    assert n % 128 == 0, "host image size must be a multiple of 128"
    a = torch.from_numpy(np.ascontiguousarray(image.a_bits[: n // 8])).cuda()
    v = torch.from_numpy(np.ascontiguousarray(image.v)).cuda()
    return a, v


def sorted_table(table: S.AllocTable):
    order = np.argsort(table.base, kind="stable")
    return table.base[order], table.size[order]


def make_pair(image: S.HostImage, table: S.AllocTable | None = None, carry: bool = True,
              strict: bool = False, **cfg):
    """A libcg Context and an oracle over the same image and table (frees
    applied to both, verdicts compared)."""
    import paper_1310_0901_gb300 as cg
    ctx = cg.Context(carry=carry, strict=strict, **cfg)
    a, v = image_tensors(image)
    ctx.bind_host_shadow(a, v)
    orc = O.Oracle(image.a_bits, image.v, carry=carry, strict=strict)
    if table is not None:
        bases, sizes = sorted_table(table)
        st = ctx.register_allocs(bases, sizes)
        assert not st.any(), st[st != 0][:5]
        for b, s in zip(bases, sizes):
            assert orc.register_alloc(int(b), int(s)) == 0
        for j in table.freed:
            b = int(table.base[j])
            assert ctx.free(b) == orc.free(b) == "OK"
    return ctx, orc, (a, v)


def assert_same_report(g: dict, o: dict, what=""):
    if g != o:
        diff = {k: (g[k], o[k]) for k in o if g.get(k) != o[k]}
        raise AssertionError(f"{what}: report differs (gpu, oracle): {diff}")


def reports_from_array(arr: np.ndarray) -> list[dict]:
    names = arr.dtype.names
    return [{k: int(r[k]) for k in names} for r in arr]


def assert_same_state(ctx, orc, v_tensor, table: S.AllocTable | None):
    """Host V image and the device shadow of every live allocation agree."""
    gv = v_tensor.cpu().numpy()
    ov = orc.read_host_v()
    if not np.array_equal(gv, ov):
        bad = np.nonzero(gv != ov)[0]
        raise AssertionError(f"host V differs at {bad[:10]} (of {bad.size})")
    if table is None:
        return
    freed = set(int(j) for j in table.freed)
    for j in range(len(table.base)):
        if j in freed:
            continue
        b, s = int(table.base[j]), int(table.size[j])
        g = ctx.read_device_shadow(b, s)
        o = orc.read_dev_v(b, s)
        if not np.array_equal(g, o):
            bad = np.nonzero(g != o)[0]
            raise AssertionError(f"device shadow of allocation {j} differs at {bad[:10]}")

"""The CPU oracle against what the paper and mathematics fix (no GPU).

Each pin lives in ``tests/pins.py`` so the mutation tests can run the same
pins against oracles with planted mistakes."""
import pytest

import oracle as O
from tests import pins


@pytest.fixture(scope="module")
def lib():
    return O.load()


@pytest.mark.parametrize("pin", pins.ALL_PINS, ids=lambda p: p.__name__)
def test_pin(lib, pin):
    pin(lib)


def test_batch_is_sequential_application(lib):
    """A batch gives the same reports and final state as the same requests
    checked one by one in order."""
    import cg_synth as S
    import numpy as np
    w = S.small(1)
    a = O.Oracle(w.image.a_bits, w.image.v, lib=lib)
    b = O.Oracle(w.image.a_bits, w.image.v, lib=lib)
    for o in (a, b):
        for base, size in zip(w.table.base, w.table.size):
            assert o.register_alloc(int(base), int(size)) == 0
        for j in w.table.freed:
            assert o.free(int(w.table.base[j])) == "OK"
    st, reps, _ = a.check_batch(w.reqs)
    assert st == 0
    for i, r in enumerate(w.reqs):
        st, rep = b.check_copy(int(r["kind"]), int(r["dst"]), int(r["src"]), int(r["n"]))
        assert st == 0 and rep == reps[i], i
    assert np.array_equal(a.read_host_v(), b.read_host_v())

"""libcg's host code built with AddressSanitizer and UndefinedBehaviorSanitizer
(`-fsanitize=address,undefined` for the host compiler): the host-only entry
points (the level planner on random batches, against the pairwise
definition; configuration defaults; report formatting) run clean.  CPU only;
the device code is the same build's."""
from __future__ import annotations

import os
import subprocess
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402  (only for its scratch directories)

CHILD = r'''
import sys, ctypes
sys.path.insert(0, sys.argv[1])
import numpy as np
import cg_synth as S
import paper_1310_0901_gb300 as cg
from tests.test_abi import _brute_levels
for seed in range(4):
    rng = np.random.default_rng(seed)
    n = 300
    reqs = np.zeros(n, S.REQ_DTYPE)
    reqs["kind"] = rng.integers(1, 4, n)
    reqs["n"] = rng.integers(0, 40, n)
    reqs["dst"] = rng.integers(0, 400, n)
    reqs["src"] = rng.integers(0, 400, n)
    modes = rng.integers(0, 4, n).astype(np.uint8)
    assert cg.plan_levels(reqs, carry=True)[0].tolist() == _brute_levels(reqs)
    assert cg.plan_levels(reqs, carry=True, modes=modes)[0].tolist() == _brute_levels(reqs, modes)
w = S.small(0)
assert cg.plan_levels(w.reqs, carry=True)[0].tolist() == _brute_levels(w.reqs)
c = cg.cg_config()
assert cg.cg_config_default(ctypes.byref(c)) == 0
rep = {f: 0 for f in cg.REPORT_FIELDS}
rep.update(flags=cg.FLAGS["OVERRUN_SRC"] | cg.FLAGS["HOST_UNADDR"], expected=8000000,
           found_src=4000000, n_unaddr=3, first_unaddr_off=7)
assert "8000000" in cg.format_report(rep, cg.DTOH)
print("HOST CLEAN")
'''


def _runtime(name: str) -> str | None:
    p = subprocess.run(["gcc", f"-print-file-name={name}"], capture_output=True, text=True)
    path = p.stdout.strip()
    return path if p.returncode == 0 and os.path.isabs(path) and os.path.exists(path) else None


@pytest.mark.timeout(900)
def test_host_code_under_asan_and_ubsan():
    asan = _runtime("libasan.so")
    if asan is None:
        pytest.skip("no AddressSanitizer runtime for gcc here")
    sys.path.insert(0, ROOT)
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "cg_build", os.path.join(ROOT, "paper_1310_0901_gb300", "build.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    d = O.scratch_dir("cg_san_")
    lib = b.build(out=os.path.join(d, "libcg.so"), obj_dir=d,
                  host_flags=("-fsanitize=address", "-fsanitize=undefined",
                              "-fno-sanitize-recover=all", "-fno-omit-frame-pointer"))
    env = dict(os.environ, LD_PRELOAD=asan, CG_LIB_PATH=lib,
               ASAN_OPTIONS="detect_leaks=0:protect_shadow_gap=0:abort_on_error=1",
               UBSAN_OPTIONS="print_stacktrace=1:halt_on_error=1")
    p = subprocess.run([sys.executable, "-c", CHILD, ROOT], env=env, capture_output=True,
                       text=True, timeout=800, cwd=ROOT)
    out = p.stdout + p.stderr
    assert p.returncode == 0 and "HOST CLEAN" in out, out[-3000:]
    assert "runtime error" not in out and "AddressSanitizer" not in out, out[-3000:]

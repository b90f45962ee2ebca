"""The oracle built with AddressSanitizer and UndefinedBehaviorSanitizer
runs every pin cleanly: no out-of-bounds access, use after free, overflow
of signed arithmetic or misaligned access in the checker the GPU path is
compared with.  CPU only."""
from __future__ import annotations

import os
import subprocess
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402


def _runtime(name: str) -> str | None:
    p = subprocess.run(["gcc", f"-print-file-name={name}"], capture_output=True, text=True)
    path = p.stdout.strip()
    return path if p.returncode == 0 and os.path.isabs(path) and os.path.exists(path) else None


@pytest.mark.timeout(900)
def test_pins_pass_under_asan_and_ubsan():
    asan = _runtime("libasan.so")
    if asan is None:
        pytest.skip("no AddressSanitizer runtime for gcc here")
    d = O.scratch_dir("cg_oracle_san_")
    lib = O.build(O.SRC, os.path.join(d, "libcg_oracle.so"), sanitize=True)
    env = dict(os.environ, LD_PRELOAD=asan,
               ASAN_OPTIONS="detect_leaks=0:abort_on_error=1",
               UBSAN_OPTIONS="print_stacktrace=1:halt_on_error=1")
    p = subprocess.run([sys.executable, os.path.join(HERE, "pins.py"), lib], env=env,
                       capture_output=True, text=True, timeout=800)
    out = p.stdout + p.stderr
    assert p.returncode == 0 and "ALL PINS PASS" in out, out[-3000:]
    assert "runtime error" not in out and "AddressSanitizer" not in out, out[-3000:]

"""Plain CPU oracle for the Cudagrind transfer checks (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  The GPU library never loads it, and it shares
no code with the GPU library: the C source (``cg_oracle.c``) keeps its own
definitions, and this binding declares its own ctypes structures.

The checker follows the paper's Sec. 2 itemize (unallocated device memory,
undefined host data sent to the device, copies larger than the allocation),
Listing 5 (expected vs found bytes), Sec. 1.1 (bit-precise A/V shadow) and
Sec. 5 (definedness tracked through all three copy directions).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "cg_oracle.c")
LIB = os.path.join(HERE, "libcg_oracle.so")

HTOD, DTOH, DTOD = 1, 2, 3
BYTE_GOOD, BYTE_UNADDR, BYTE_UNDEF = 0, 1, 2
FLAG_NAMES = [
    "UNALLOC_DST", "UNALLOC_SRC", "OVERRUN_DST", "OVERRUN_SRC",
    "HOST_UNADDR", "HOST_UNDEF", "DEV_UNDEF_SRC", "DTOD_OVERLAP", "CONCURRENT",
]
FLAGS = {name: 1 << i for i, name in enumerate(FLAG_NAMES)}
FREE_NAMES = {0: "OK", 1: "UNKNOWN", 2: "DOUBLE", 3: "INTERIOR"}
STATUS = {0: "OK", -1: "E_ARG", -2: "E_KIND", -3: "E_HOST_RANGE",
          -4: "E_ZERO_SIZE", -5: "E_WRAP", -6: "E_OVERLAP", -7: "E_NOMEM",
          -8: "E_RANGE"}
STATUS_CODES = {name: code for code, name in STATUS.items()}
ARG_READ, ARG_WRITE = 1, 2


class OrReport(ctypes.Structure):
    _fields_ = [
        ("flags", ctypes.c_uint32), ("first_bad_kind", ctypes.c_uint32),
        ("first_bad_off", ctypes.c_int64), ("first_unaddr_off", ctypes.c_int64),
        ("first_undef_off", ctypes.c_int64), ("n_good", ctypes.c_uint64),
        ("n_unaddr", ctypes.c_uint64), ("n_undef", ctypes.c_uint64),
        ("expected", ctypes.c_uint64), ("found_dst", ctypes.c_uint64),
        ("found_src", ctypes.c_uint64), ("alloc_base_dst", ctypes.c_uint64),
        ("alloc_size_dst", ctypes.c_uint64), ("alloc_base_src", ctypes.c_uint64),
        ("alloc_size_src", ctypes.c_uint64), ("race_seq", ctypes.c_int64),
    ]


class OrSide3d(ctypes.Structure):
    _fields_ = [
        ("ptr", ctypes.c_uint64), ("pitch", ctypes.c_uint64), ("rows", ctypes.c_uint64),
        ("x", ctypes.c_uint64), ("y", ctypes.c_uint64), ("z", ctypes.c_uint64),
        ("is_array", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
    ]


class OrCopy3d(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
        ("dst", OrSide3d), ("src", OrSide3d),
        ("width", ctypes.c_uint64), ("height", ctypes.c_uint64), ("depth", ctypes.c_uint64),
    ]


def side(ptr: int, pitch: int = 0, rows: int = 0, x: int = 0, y: int = 0, z: int = 0,
         array: bool = False) -> dict:
    """One side of a pitched copy (see or_check_copy3d)."""
    return dict(ptr=ptr, pitch=pitch, rows=rows, x=x, y=y, z=z, is_array=int(array))


class OrRecord(ctypes.Structure):
    _fields_ = [
        ("req", ctypes.c_uint64), ("cls", ctypes.c_uint32),
        ("severity", ctypes.c_uint32), ("off", ctypes.c_int64),
        ("count", ctypes.c_uint64), ("expected", ctypes.c_uint64),
        ("found", ctypes.c_uint64),
    ]


REPORT_FIELDS = [f for f, _ in OrReport._fields_]
RECORD_FIELDS = [f for f, _ in OrRecord._fields_]


def build(src: str = SRC, out: str = LIB, werror: bool = True, sanitize: bool = False) -> str:
    """Compile the oracle with plain gcc (no vector intrinsics, portable).
    sanitize: an AddressSanitizer + UndefinedBehaviorSanitizer build (load
    it in a process started with the ASan runtime preloaded)."""
    cmd = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-Wall", "-Wextra"]
    cmd += ["-Werror"] if werror else []
    if sanitize:
        cmd += ["-g", "-fno-omit-frame-pointer", "-fsanitize=address,undefined",
                "-fno-sanitize-recover=all"]
    cmd += ["-o", out, src]
    subprocess.run(cmd, check=True)
    return out


def _needs_build(lib: str, src: str) -> bool:
    if not os.path.exists(lib):
        return True
    hdr = os.path.join(os.path.dirname(src), "cg_oracle.h")
    newest = max(os.path.getmtime(src), os.path.getmtime(hdr) if os.path.exists(hdr) else 0)
    return os.path.getmtime(lib) < newest


def load(path: str | None = None) -> ctypes.CDLL:
    """Load (building first if stale) the oracle shared library."""
    if path is None:
        path = LIB
        if _needs_build(path, SRC):
            build(SRC, path)
    lib = ctypes.CDLL(path)
    u64, i32, u32, vp = ctypes.c_uint64, ctypes.c_int, ctypes.c_uint32, ctypes.c_void_p
    lib.or_create.restype = vp
    lib.or_create.argtypes = [u64, vp, vp, i32, i32]
    lib.or_destroy.argtypes = [vp]
    lib.or_destroy.restype = None
    lib.or_register_alloc.argtypes = [vp, u64, u64]
    lib.or_register_alloc.restype = i32
    lib.or_register_allocs.argtypes = [vp, vp, vp, u64, vp]
    lib.or_register_allocs.restype = u64
    lib.or_free.argtypes = [vp, u64, ctypes.POINTER(u32)]
    lib.or_free.restype = i32
    lib.or_mark.argtypes = [vp, u64, u64, ctypes.c_uint8]
    lib.or_mark.restype = i32
    lib.or_check_copy.argtypes = [vp, u32, u64, u64, u64, ctypes.POINTER(OrReport)]
    lib.or_check_copy.restype = i32
    lib.or_check_batch.argtypes = [vp, vp, vp, vp, vp, u64, vp, ctypes.POINTER(u64)]
    lib.or_check_batch.restype = i32
    lib.or_emit_records.argtypes = [vp, vp, vp, vp, vp, u64, i32, vp, u64]
    lib.or_emit_records.restype = u64
    lib.or_read_host_v.argtypes = [vp, u64, u64, vp]
    lib.or_read_host_v.restype = i32
    lib.or_read_dev_v.argtypes = [vp, u64, u64, vp]
    lib.or_read_dev_v.restype = i32
    lib.or_live_count.argtypes = [vp]
    lib.or_live_count.restype = u64
    lib.or_memset.argtypes = [vp, u64, u64, u64, u64, ctypes.POINTER(OrReport)]
    lib.or_memset.restype = i32
    lib.or_check_kernel_args.argtypes = [vp, vp, vp, vp, u64, vp]
    lib.or_check_kernel_args.restype = i32
    lib.or_check_copy3d.argtypes = [vp, ctypes.POINTER(OrCopy3d), ctypes.POINTER(OrReport)]
    lib.or_check_copy3d.restype = i32
    lib.or_register_array.argtypes = [vp, u64, u64, u64, u64]
    lib.or_register_array.restype = i32
    lib.or_free_array.argtypes = [vp, u64, ctypes.POINTER(u32)]
    lib.or_free_array.restype = i32
    lib.or_read_array_v.argtypes = [vp, u64, u64, u64, vp]
    lib.or_read_array_v.restype = i32
    lib.or_races.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, u64, vp]
    lib.or_races.restype = u64
    return lib


SCRATCH = os.path.join(os.path.dirname(HERE), "_build", "tmp")  # git-ignored


def scratch_dir(prefix: str) -> str:
    """A fresh directory for build artefacts of the tests, inside the
    repository's git-ignored build folder."""
    os.makedirs(SCRATCH, exist_ok=True)
    return tempfile.mkdtemp(prefix=prefix, dir=SCRATCH)


def build_variant(source_text: str, tag: str) -> str:
    """Compile a modified copy of the oracle source (used by the mutation
    tests, which plant a mistake in the oracle and expect a pin to fail)."""
    d = scratch_dir(f"cg_oracle_{tag}_")
    with open(os.path.join(d, "cg_oracle.h"), "w") as f:
        f.write(open(os.path.join(HERE, "cg_oracle.h")).read())
    src = os.path.join(d, "cg_oracle.c")
    with open(src, "w") as f:
        f.write(source_text)
    return build(src, os.path.join(d, "libcg_oracle.so"), werror=False)


def report_dict(r: OrReport) -> dict:
    return {f: getattr(r, f) for f in REPORT_FIELDS}


def _u8ptr(a: np.ndarray) -> int:
    assert a.dtype == np.uint8 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


class Oracle:
    """A checker state: host shadow image, live allocations, device shadow."""

    def __init__(self, a_bits: np.ndarray, v: np.ndarray, carry: bool = True,
                 strict: bool = False, lib: ctypes.CDLL | None = None):
        self.lib = lib if lib is not None else load()
        v = np.ascontiguousarray(v, dtype=np.uint8)
        a_bits = np.ascontiguousarray(a_bits, dtype=np.uint8)
        assert a_bits.size >= (v.size + 7) // 8
        self.host_n = int(v.size)
        self.strict = bool(strict)
        self._h = self.lib.or_create(self.host_n, _u8ptr(a_bits) if a_bits.size else None,
                                     _u8ptr(v) if v.size else None, int(carry), int(strict))
        if not self._h:
            raise MemoryError("oracle state allocation failed")

    def close(self):
        if self._h:
            self.lib.or_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def register_alloc(self, base: int, size: int) -> int:
        return self.lib.or_register_alloc(self._h, base, size)

    def register_allocs(self, bases, sizes) -> np.ndarray:
        """register_alloc for each (base, size) in turn; the statuses."""
        b = np.ascontiguousarray(bases, dtype=np.uint64)
        z = np.ascontiguousarray(sizes, dtype=np.uint64)
        st = np.zeros(max(1, len(b)), dtype=np.int32)
        self.lib.or_register_allocs(self._h, b.ctypes.data, z.ctypes.data, len(b), st.ctypes.data)
        return st[:len(b)]

    def free(self, base: int) -> str:
        v = ctypes.c_uint32(99)
        st = self.lib.or_free(self._h, base, ctypes.byref(v))
        assert st == 0, st
        return FREE_NAMES[v.value]

    def mark(self, dptr: int, n: int, value: int) -> int:
        return self.lib.or_mark(self._h, dptr, n, value)

    def check_copy(self, kind: int, dst: int, src: int, n: int):
        r = OrReport()
        st = self.lib.or_check_copy(self._h, kind, dst, src, n, ctypes.byref(r))
        return st, report_dict(r)

    def check_copy3d(self, kind: int, dst: dict, src: dict, width: int, height: int,
                     depth: int = 1):
        q = OrCopy3d(kind=kind, reserved=0, dst=OrSide3d(reserved=0, **dst),
                     src=OrSide3d(reserved=0, **src), width=width, height=height, depth=depth)
        r = OrReport()
        st = self.lib.or_check_copy3d(self._h, ctypes.byref(q), ctypes.byref(r))
        return st, report_dict(r)

    def memset(self, dptr: int, width: int, height: int = 1, pitch: int = 0):
        r = OrReport()
        st = self.lib.or_memset(self._h, dptr, pitch, width, height, ctypes.byref(r))
        return st, report_dict(r)

    def check_kernel_args(self, ptr, nbytes, access):
        """Arguments as three sequences; returns (status, list of report dicts)."""
        p = np.ascontiguousarray(ptr, dtype=np.uint64)
        b = np.ascontiguousarray(nbytes, dtype=np.uint64)
        a = np.ascontiguousarray(access, dtype=np.uint32)
        n = len(p)
        reps = (OrReport * max(1, n))()
        st = self.lib.or_check_kernel_args(self._h, p.ctypes.data, b.ctypes.data, a.ctypes.data,
                                           n, reps)
        return st, [report_dict(reps[i]) for i in range(n)]

    def register_array(self, handle: int, w: int, h: int, d: int = 1) -> int:
        return self.lib.or_register_array(self._h, handle, w, h, d)

    def free_array(self, handle: int) -> str:
        v = ctypes.c_uint32(99)
        st = self.lib.or_free_array(self._h, handle, ctypes.byref(v))
        assert st == 0, st
        return FREE_NAMES[v.value]

    def read_array_v(self, handle: int, off: int, n: int) -> np.ndarray:
        out = np.empty(n, dtype=np.uint8)
        st = self.lib.or_read_array_v(self._h, handle, off, n, out.ctypes.data if n else None)
        assert st == 0, st
        return out

    def check_batch(self, reqs: np.ndarray):
        """reqs: structured array with fields kind, dst, src, n."""
        k = np.ascontiguousarray(reqs["kind"], dtype=np.uint32)
        d = np.ascontiguousarray(reqs["dst"], dtype=np.uint64)
        s = np.ascontiguousarray(reqs["src"], dtype=np.uint64)
        n = np.ascontiguousarray(reqs["n"], dtype=np.uint64)
        reps = (OrReport * max(1, len(reqs)))()
        bad = ctypes.c_uint64(0)
        st = self.lib.or_check_batch(self._h, k.ctypes.data, d.ctypes.data, s.ctypes.data,
                                     n.ctypes.data, len(reqs), ctypes.addressof(reps),
                                     ctypes.byref(bad))
        return st, [report_dict(reps[i]) for i in range(len(reqs))], int(bad.value)

    def check_copy_status(self, kind: int, dst: int, src: int, n: int) -> int:
        """check_copy without building the report dict (for timing)."""
        if not hasattr(self, "_rep"):
            self._rep = OrReport()
            self._rep_ref = ctypes.byref(self._rep)
        return self.lib.or_check_copy(self._h, kind, dst, src, n, self._rep_ref)

    def batch_runner(self, reqs: np.ndarray):
        """A callable that applies the batch `reqs` (or_check_batch) and
        returns its status, with no report dicts built (for timing)."""
        arrs = [np.ascontiguousarray(reqs[f], dtype=t) for f, t in
                (("kind", np.uint32), ("dst", np.uint64), ("src", np.uint64), ("n", np.uint64))]
        reps = (OrReport * max(1, len(reqs)))()
        bad = ctypes.c_uint64(0)
        ptrs = [a.ctypes.data for a in arrs]

        def run() -> int:
            return self.lib.or_check_batch(self._h, *ptrs, len(reqs), ctypes.addressof(reps),
                                           ctypes.byref(bad))
        run.keep = (arrs, reps, bad)
        return run

    def read_host_v(self, off: int = 0, n: int | None = None) -> np.ndarray:
        n = self.host_n - off if n is None else n
        out = np.empty(n, dtype=np.uint8)
        st = self.lib.or_read_host_v(self._h, off, n, out.ctypes.data if n else None)
        assert st == 0, st
        return out

    def read_dev_v(self, dptr: int, n: int) -> np.ndarray:
        out = np.empty(n, dtype=np.uint8)
        st = self.lib.or_read_dev_v(self._h, dptr, n, out.ctypes.data if n else None)
        assert st == 0, st
        return out

    def live_count(self) -> int:
        return int(self.lib.or_live_count(self._h))


def emit_records(reports: list[dict], reqs: np.ndarray, strict: bool = False,
                 lib: ctypes.CDLL | None = None) -> list[dict]:
    lib = lib if lib is not None else load()
    nreq = len(reqs)
    reps = (OrReport * max(1, nreq))()
    for i, r in enumerate(reports):
        for f in REPORT_FIELDS:
            setattr(reps[i], f, r[f])
    k = np.ascontiguousarray(reqs["kind"], dtype=np.uint32)
    d = np.ascontiguousarray(reqs["dst"], dtype=np.uint64)
    s = np.ascontiguousarray(reqs["src"], dtype=np.uint64)
    n = np.ascontiguousarray(reqs["n"], dtype=np.uint64)
    total = lib.or_emit_records(ctypes.addressof(reps), k.ctypes.data, d.ctypes.data,
                                s.ctypes.data, n.ctypes.data, nreq, int(strict), None, 0)
    out = (OrRecord * max(1, total))()
    lib.or_emit_records(ctypes.addressof(reps), k.ctypes.data, d.ctypes.data, s.ctypes.data,
                        n.ctypes.data, nreq, int(strict), ctypes.addressof(out), total)
    return [{f: getattr(out[i], f) for f in RECORD_FIELDS} for i in range(total)]


def races(reqs: np.ndarray, client: np.ndarray, submit_ns: np.ndarray, done_ns: np.ndarray,
          moved: np.ndarray, lib: ctypes.CDLL | None = None) -> np.ndarray:
    """race_seq per request of a served trace given in seq order (see or_races)."""
    lib = lib if lib is not None else load()
    n = len(reqs)
    k = np.ascontiguousarray(reqs["kind"], dtype=np.uint32)
    d = np.ascontiguousarray(reqs["dst"], dtype=np.uint64)
    s = np.ascontiguousarray(reqs["src"], dtype=np.uint64)
    nn = np.ascontiguousarray(reqs["n"], dtype=np.uint64)
    c = np.ascontiguousarray(client, dtype=np.uint32)
    sub = np.ascontiguousarray(submit_ns, dtype=np.uint64)
    done = np.ascontiguousarray(done_ns, dtype=np.uint64)
    mv = np.ascontiguousarray(moved, dtype=np.uint8)
    out = np.full(max(1, n), -1, dtype=np.int64)
    lib.or_races(k.ctypes.data, d.ctypes.data, s.ctypes.data, nn.ctypes.data, c.ctypes.data,
                 sub.ctypes.data, done.ctypes.data, mv.ctypes.data, n, out.ctypes.data)
    return out[:n]

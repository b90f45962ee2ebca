"""Python binding of libcg (``include/cg.h``): GPU transfer checks in the
manner of Cudagrind (Baumann & Gracia, 2013).

Argument marshalling only: every check runs in libcg's CUDA kernels.  The
shared library is built in-tree by ``paper_1310_0901_gb300.build.build()``;
importing this package without it raises, so there is no silent fallback.

The C entry points are exposed under their own names (``cg_create``,
``cg_check_copy``, ...) with ctypes signatures; ``Context`` wraps them for
torch tensors (device memory) and numpy request arrays.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
# CG_LIB_PATH selects another build of the same library (an instrumented one)
LIB_PATH = os.environ.get("CG_LIB_PATH") or os.path.join(PKG, "libcg.so")

HTOD, DTOH, DTOD = 1, 2, 3
BYTE_GOOD, BYTE_UNADDR, BYTE_UNDEF = 0, 1, 2
FLAG_NAMES = ["UNALLOC_DST", "UNALLOC_SRC", "OVERRUN_DST", "OVERRUN_SRC",
              "HOST_UNADDR", "HOST_UNDEF", "DEV_UNDEF_SRC", "DTOD_OVERLAP", "CONCURRENT"]
FLAGS = {n: 1 << i for i, n in enumerate(FLAG_NAMES)}
FREE_NAMES = {0: "OK", 1: "UNKNOWN", 2: "DOUBLE", 3: "INTERIOR"}
STATUS = {0: "OK", -1: "E_ARG", -2: "E_KIND", -3: "E_HOST_RANGE", -4: "E_ZERO_SIZE",
          -5: "E_WRAP", -6: "E_OVERLAP", -7: "E_NOMEM", -8: "E_RANGE", -9: "E_CUDA",
          -10: "E_NO_HOST", -11: "E_ALIGN", -12: "E_STATE", -13: "E_TIMEOUT",
          -14: "E_FULL", -15: "E_TOO_BIG"}

u32, u64, i32, i64, vp = (ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int32, ctypes.c_int64,
                          ctypes.c_void_p)


class cg_copy(ctypes.Structure):
    _fields_ = [("kind", u32), ("reserved", u32), ("dst", u64), ("src", u64), ("n", u64)]


class cg_karg(ctypes.Structure):
    _fields_ = [("ptr", u64), ("bytes", u64), ("access", u32), ("reserved", u32)]


ARG_READ, ARG_WRITE = 1, 2
FAULT_STALL_COPY, FAULT_SHADOW_ALLOC = 1, 2
KARG_DTYPE = np.dtype([("ptr", "<u8"), ("bytes", "<u8"), ("access", "<u4"), ("reserved", "<u4")])


class cg_side3d(ctypes.Structure):
    _fields_ = [("ptr", u64), ("pitch", u64), ("rows", u64), ("x", u64), ("y", u64),
                ("z", u64), ("is_array", u32), ("reserved", u32)]


class cg_copy3d(ctypes.Structure):
    _fields_ = [("kind", u32), ("reserved", u32), ("dst", cg_side3d), ("src", cg_side3d),
                ("width", u64), ("height", u64), ("depth", u64)]


def side(ptr: int, pitch: int = 0, rows: int = 0, x: int = 0, y: int = 0, z: int = 0,
         array: bool = False) -> dict:
    """One side of a pitched copy: a device address, a host offset, or (with
    array=True) a device array's handle; pitch = bytes between rows, rows =
    rows per slice, (x, y, z) = origin with x in bytes."""
    return dict(ptr=ptr, pitch=pitch, rows=rows, x=x, y=y, z=z, is_array=int(array))


def copy3d(kind: int, dst: dict, src: dict, width: int, height: int, depth: int = 1) -> cg_copy3d:
    return cg_copy3d(kind=kind, reserved=0, dst=cg_side3d(reserved=0, **dst),
                     src=cg_side3d(reserved=0, **src), width=width, height=height, depth=depth)


class cg_report(ctypes.Structure):
    _fields_ = [("flags", u32), ("first_bad_kind", u32), ("first_bad_off", i64),
                ("first_unaddr_off", i64), ("first_undef_off", i64), ("n_good", u64),
                ("n_unaddr", u64), ("n_undef", u64), ("expected", u64), ("found_dst", u64),
                ("found_src", u64), ("alloc_base_dst", u64), ("alloc_size_dst", u64),
                ("alloc_base_src", u64), ("alloc_size_src", u64), ("race_seq", i64)]


class cg_err_record(ctypes.Structure):
    _fields_ = [("req", u64), ("cls", u32), ("severity", u32), ("off", i64), ("count", u64),
                ("expected", u64), ("found", u64)]


class cg_config(ctypes.Structure):
    _fields_ = [("carry", u32), ("strict_device_undef", u32), ("shadow_slab_bytes", u64),
                ("shadow_budget_bytes", u64), ("scan_ctas_per_sm", u32),
                ("batch_segment_kib", u32), ("batch_ctas_per_sm", u32),
                ("scan_engine", u32), ("batch_autotune", u32), ("batch_direct_launch", u32),
                ("batch_piece_kib", u32), ("reserved", u32 * 5)]


class cg_stats(ctypes.Structure):
    _fields_ = [("checks", u64), ("bytes_checked", u64), ("batches", u64), ("levels", u64),
                ("kernels", u64), ("errors", u64 * 9), ("live_allocs", u64),
                ("shadow_bytes", u64), ("batch_ns", u64), ("batch_plan_ns", u64),
                ("batch_lookup_ns", u64), ("table_uploads", u64), ("table_merges", u64)]


class cg_request(ctypes.Structure):
    _fields_ = [("op", u32), ("kind", u32), ("dst", u64), ("src", u64), ("n", u64)]


class cg_result(ctypes.Structure):
    _fields_ = [("seq", u64), ("status", i32), ("verdict", u32), ("submit_ns", u64),
                ("done_ns", u64), ("report", cg_report)]


class cg_serve_config(ctypes.Structure):
    _fields_ = [("clients", u32), ("ring_capacity", u32), ("max_round", u32), ("streams", u32),
                ("budget_bytes", u64), ("reserved", u32 * 10)]


class cg_serve_stats(ctypes.Structure):
    _fields_ = [("requests", u64), ("checks", u64), ("rounds", u64), ("round_checks_max", u64),
                ("conflict_waits", u64), ("budget_stalls", u64), ("bytes_checked", u64),
                ("inflight_bytes_max", u64)]


OP_CHECK, OP_ALLOC, OP_FREE, OP_MARK_DEFINED, OP_MARK_UNDEFINED = 1, 2, 3, 4, 5
PENDING = 1
REQUEST_DTYPE = np.dtype([("op", "<u4"), ("kind", "<u4"), ("dst", "<u8"), ("src", "<u8"),
                          ("n", "<u8")])

REPORT_FIELDS = [f for f, _ in cg_report._fields_]
RECORD_FIELDS = [f for f, _ in cg_err_record._fields_]
REPORT_DTYPE = np.dtype([(f, "<i8" if t is i64 else ("<u4" if t is u32 else "<u8"))
                         for f, t in cg_report._fields_])
RECORD_DTYPE = np.dtype([(f, "<i8" if t is i64 else ("<u4" if t is u32 else "<u8"))
                         for f, t in cg_err_record._fields_])
RESULT_DTYPE = np.dtype([("seq", "<u8"), ("status", "<i4"), ("verdict", "<u4"),
                         ("submit_ns", "<u8"), ("done_ns", "<u8"), ("report", REPORT_DTYPE)])
assert ctypes.sizeof(cg_copy) == 32 and ctypes.sizeof(cg_report) == 120
assert ctypes.sizeof(cg_err_record) == 48
assert ctypes.sizeof(cg_request) == 32 and ctypes.sizeof(cg_result) == 152
assert REPORT_DTYPE.itemsize == 120 and RECORD_DTYPE.itemsize == 48

# (name, restype, argtypes) of every entry point declared in include/cg.h
SIGNATURES = [
    ("cg_config_default", i32, [ctypes.POINTER(cg_config)]),
    ("cg_create", i32, [ctypes.POINTER(vp), ctypes.POINTER(cg_config)]),
    ("cg_destroy", i32, [vp]),
    ("cg_bind_host_shadow", i32, [vp, vp, vp, u64]),
    ("cg_upload_host_shadow", i32, [vp, vp, vp, u64, u64, vp]),
    ("cg_register_alloc", i32, [vp, u64, u64]),
    ("cg_register_allocs", i32, [vp, vp, vp, u64, vp]),
    ("cg_free", i32, [vp, u64, ctypes.POINTER(u32)]),
    ("cg_mark_defined", i32, [vp, u64, u64, vp]),
    ("cg_mark_undefined", i32, [vp, u64, u64, vp]),
    ("cg_read_device_shadow", i32, [vp, u64, u64, vp]),
    ("cg_check_copy", i32, [vp, ctypes.POINTER(cg_copy), ctypes.POINTER(cg_report), vp]),
    ("cg_check_copy_async", i32, [vp, ctypes.POINTER(cg_copy), vp, vp]),
    ("cg_check_batch", i32, [vp, vp, u64, vp, vp, u64, ctypes.POINTER(u64),
                             ctypes.POINTER(u64), vp]),
    ("cg_serve_start", i32, [vp, ctypes.POINTER(cg_serve_config)]),
    ("cg_submit", i32, [vp, u32, ctypes.POINTER(cg_request), ctypes.POINTER(u64)]),
    ("cg_poll", i32, [vp, u64, ctypes.POINTER(cg_result)]),
    ("cg_wait", i32, [vp, u64, u32, ctypes.POINTER(cg_result)]),
    ("cg_serve_replay", i32, [vp, vp, vp, vp, u64, vp]),
    ("cg_serve_stop", i32, [vp, ctypes.POINTER(cg_serve_stats)]),
    ("cg_plan_units", i32, [vp, u64, u32, vp, u64, u64, vp, vp, vp, vp, u64, vp]),
    ("cg_scan_noalloc", i32, [u32, vp, vp, u64, u64, vp, vp, u64, u32, vp, vp]),
    ("cg_check_batch_async", i32, [vp, vp, u64, u64, ctypes.POINTER(u64), ctypes.POINTER(u64),
                                   vp]),
    ("cg_batch_wait", i32, [vp, u64, vp, vp, u64, ctypes.POINTER(u64)]),
    ("cg_get_tuned", i32, [vp, vp, vp, u32, ctypes.POINTER(u32)]),
    ("cg_add_tuned", i32, [vp, vp, vp, u32]),
    ("cg_inject_fault", i32, [vp, u32]),
    ("cg_snapshot", i32, [vp, ctypes.c_char_p]),
    ("cg_restore", i32, [vp, ctypes.c_char_p]),
    ("cg_check_memset", i32, [vp, u64, u64, u64, u64, vp, vp]),
    ("cg_check_memset_async", i32, [vp, u64, u64, u64, u64, vp, vp]),
    ("cg_check_kernel_args", i32, [vp, vp, u64, vp, ctypes.POINTER(u64), vp]),
    ("cg_register_array", i32, [vp, u64, u64, u64, u64]),
    ("cg_free_array", i32, [vp, u64, ctypes.POINTER(u32)]),
    ("cg_read_array_shadow", i32, [vp, u64, u64, u64, vp]),
    ("cg_check_copy3d", i32, [vp, ctypes.POINTER(cg_copy3d), vp, vp]),
    ("cg_check_copy3d_async", i32, [vp, ctypes.POINTER(cg_copy3d), vp, vp]),
    ("cg_batch_features", i32, [vp, u64, vp]),
    ("cg_tune_batch", i32, [vp, vp, u64, vp, u32, u32, u32, vp, ctypes.POINTER(u32), vp]),
    ("cg_set_cost_model", i32, [vp, vp, u32]),
    ("cg_mlp_fit", i32, [vp, vp, u32, u32, u32, ctypes.c_float, u64, vp, vp, vp]),
    ("cg_mlp_grad", i32, [vp, vp, u32, u32, vp, vp, ctypes.POINTER(ctypes.c_float), vp]),
    ("cg_choose_segment", i32, [vp, vp, u64, ctypes.POINTER(u32), ctypes.POINTER(u32)]),
    ("cg_plan_levels", i32, [vp, u64, u32, vp, vp, ctypes.POINTER(u32)]),
    ("cg_get_stats", i32, [vp, ctypes.POINTER(cg_stats)]),
    ("cg_device_table", i32, [vp, vp, vp, vp, u64, ctypes.POINTER(u64), vp]),
    ("cg_format_report", i32, [ctypes.POINTER(cg_report), u32, ctypes.c_char_p, ctypes.c_size_t]),
    ("cg_last_error", ctypes.c_char_p, []),
    ("cg_version", ctypes.c_char_p, []),
]


def _load() -> ctypes.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"libcg.so is not built ({LIB_PATH} missing): run "
            "`python paper_1310_0901_gb300/build.py` or __graft_entry__.build()")
    lib = ctypes.CDLL(LIB_PATH)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load()
for _name, _, _ in SIGNATURES:
    globals()[_name] = getattr(_lib, _name)


class CgError(RuntimeError):
    def __init__(self, status: int, what: str):
        msg = cg_last_error().decode(errors="replace")
        super().__init__(f"{what}: {STATUS.get(status, status)} ({msg})")
        self.status = status


def check(status: int, what: str = "libcg") -> None:
    if status != 0:
        raise CgError(status, what)


def _stream_handle(stream) -> int | None:
    if stream is None:
        try:
            import torch
            return torch.cuda.current_stream().cuda_stream
        except Exception:
            return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def report_to_dict(r: cg_report) -> dict:
    return {f: getattr(r, f) for f in REPORT_FIELDS}


class Context:
    """One libcg context: allocation table, device shadow pool, bound image."""

    def __init__(self, carry: bool = True, strict: bool = False, **cfg):
        c = cg_config()
        check(cg_config_default(ctypes.byref(c)))
        c.carry = int(carry)
        c.strict_device_undef = int(strict)
        for k, v in cfg.items():
            setattr(c, k, v)
        self.cfg = c
        h = vp()
        check(cg_create(ctypes.byref(h), ctypes.byref(c)), "cg_create")
        self._h = h
        self._image = None

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            cg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def bind_host_shadow(self, a_bits, v) -> None:
        """a_bits, v: CUDA uint8 tensors (kept referenced while bound)."""
        check(cg_bind_host_shadow(self._h, a_bits.data_ptr(), v.data_ptr(), v.numel()),
              "cg_bind_host_shadow")
        self._image = (a_bits, v)

    def upload_host_shadow(self, a_host, v_host, off: int, n: int, stream=None) -> None:
        check(cg_upload_host_shadow(self._h, a_host.data_ptr(), v_host.data_ptr(), off, n,
                                    _stream_handle(stream)), "cg_upload_host_shadow")

    def register_alloc(self, dptr: int, size: int) -> int:
        return cg_register_alloc(self._h, dptr, size)

    def register_allocs(self, bases: np.ndarray, sizes: np.ndarray) -> np.ndarray:
        b = np.ascontiguousarray(bases, dtype=np.uint64)
        s = np.ascontiguousarray(sizes, dtype=np.uint64)
        st = np.zeros(len(b), dtype=np.int32)
        cg_register_allocs(self._h, b.ctypes.data, s.ctypes.data, len(b), st.ctypes.data)
        return st

    def free(self, dptr: int) -> str:
        v = u32(99)
        check(cg_free(self._h, dptr, ctypes.byref(v)), "cg_free")
        return FREE_NAMES[v.value]

    def mark_defined(self, dptr: int, n: int, stream=None) -> int:
        return cg_mark_defined(self._h, dptr, n, _stream_handle(stream))

    def mark_undefined(self, dptr: int, n: int, stream=None) -> int:
        return cg_mark_undefined(self._h, dptr, n, _stream_handle(stream))

    def read_device_shadow(self, dptr: int, n: int) -> np.ndarray:
        out = np.empty(n, dtype=np.uint8)
        check(cg_read_device_shadow(self._h, dptr, n, out.ctypes.data if n else None),
              "cg_read_device_shadow")
        return out

    def check_copy(self, kind: int, dst: int, src: int, n: int, stream=None):
        q = cg_copy(kind, 0, dst, src, n)
        r = cg_report()
        st = cg_check_copy(self._h, ctypes.byref(q), ctypes.byref(r), _stream_handle(stream))
        return st, report_to_dict(r)

    def check_copy3d(self, kind: int, dst: dict, src: dict, width: int, height: int,
                     depth: int = 1, stream=None):
        """A pitched copy (see side()); returns (status, report dict)."""
        q = copy3d(kind, dst, src, width, height, depth)
        r = cg_report()
        st = cg_check_copy3d(self._h, ctypes.byref(q), ctypes.byref(r), _stream_handle(stream))
        return st, report_to_dict(r)

    def snapshot(self, path: str) -> int:
        return cg_snapshot(self._h, os.fsencode(path))

    def restore(self, path: str) -> int:
        return cg_restore(self._h, os.fsencode(path))

    def check_memset(self, dptr: int, width: int, height: int = 1, pitch: int = 0, stream=None):
        """A memset of height rows of width bytes at dptr + y*pitch."""
        r = cg_report()
        st = cg_check_memset(self._h, dptr, pitch, width, height, ctypes.byref(r),
                             _stream_handle(stream))
        return st, report_to_dict(r)

    def check_kernel_args(self, args: np.ndarray, stream=None):
        """args: structured array of KARG_DTYPE.  Returns (status, reports as
        a structured array, bad index)."""
        args = np.ascontiguousarray(args, dtype=KARG_DTYPE)
        n = len(args)
        reps = np.zeros(max(1, n), dtype=REPORT_DTYPE)
        bad = u64(0)
        st = cg_check_kernel_args(self._h, args.ctypes.data if n else None, n, reps.ctypes.data,
                                  ctypes.byref(bad), _stream_handle(stream))
        return st, reps[:n], int(bad.value)

    def register_array(self, handle: int, width: int, height: int, depth: int = 1) -> int:
        return cg_register_array(self._h, handle, width, height, depth)

    def free_array(self, handle: int) -> str:
        v = u32(99)
        check(cg_free_array(self._h, handle, ctypes.byref(v)), "cg_free_array")
        return FREE_NAMES[v.value]

    def read_array_shadow(self, handle: int, off: int, n: int) -> np.ndarray:
        out = np.empty(n, dtype=np.uint8)
        check(cg_read_array_shadow(self._h, handle, off, n, out.ctypes.data if n else None),
              "cg_read_array_shadow")
        return out

    def check_batch_async(self, reqs: np.ndarray, rec_cap: int | None = None, stream=None):
        """Enqueue a batch; returns (status, ticket, bad index).  The request
        array is copied before return."""
        reqs = np.ascontiguousarray(reqs)
        assert reqs.dtype.itemsize == 32
        n = len(reqs)
        t = u64(0)
        bad = u64(0)
        st = cg_check_batch_async(self._h, reqs.ctypes.data, n, 8 * n if rec_cap is None else rec_cap,
                                  ctypes.byref(t), ctypes.byref(bad), _stream_handle(stream))
        return st, int(t.value), int(bad.value)

    def batch_wait(self, ticket: int, nreq: int, rec_cap: int | None = None,
                   reps_out: np.ndarray | None = None, recs_out: np.ndarray | None = None):
        """Results of an enqueued batch: (status, reports, records, total).
        reps_out / recs_out (REPORT_DTYPE / RECORD_DTYPE arrays of at least
        nreq / rec_cap entries) receive them if given; fresh arrays otherwise."""
        if rec_cap is None:
            rec_cap = 8 * nreq
        reps = reps_out if reps_out is not None else np.empty(max(1, nreq), dtype=REPORT_DTYPE)
        recs = recs_out if recs_out is not None else np.empty(max(1, rec_cap), dtype=RECORD_DTYPE)
        assert len(reps) >= nreq and len(recs) >= min(rec_cap, 1)
        n_rec = u64(0)
        st = cg_batch_wait(self._h, ticket, reps.ctypes.data, recs.ctypes.data, rec_cap,
                           ctypes.byref(n_rec))
        total = int(n_rec.value)
        return st, reps[:nreq], recs[:min(total, rec_cap)], total

    def check_batch(self, reqs: np.ndarray, rec_cap: int | None = None, stream=None,
                    reps_out: np.ndarray | None = None, recs_out: np.ndarray | None = None):
        """reqs: structured array with the layout of cg_copy (cg_synth.REQ_DTYPE).
        Returns (status, reports as a structured array, records as a
        structured array, total record count, bad index).  reps_out /
        recs_out, if given, receive the results (no fresh arrays)."""
        reqs = np.ascontiguousarray(reqs)
        assert reqs.dtype.itemsize == 32
        n = len(reqs)
        if rec_cap is None:
            rec_cap = 8 * n
        reps = reps_out[:n] if reps_out is not None else np.zeros(n, dtype=REPORT_DTYPE)
        recs = recs_out if recs_out is not None else np.zeros(max(1, rec_cap), dtype=RECORD_DTYPE)
        n_rec = u64(0)
        bad = u64(0)
        st = cg_check_batch(self._h, reqs.ctypes.data if n else None, n,
                            reps.ctypes.data if n else None,
                            recs.ctypes.data if rec_cap else None, rec_cap,
                            ctypes.byref(n_rec), ctypes.byref(bad), _stream_handle(stream))
        total = int(n_rec.value)
        return st, reps, recs[:min(total, rec_cap)], total, int(bad.value)

    # ------------------------------------------------------- batch split
    def tune_batch(self, reqs: np.ndarray, candidates=None, repeats: int = 2,
                   remember: bool = True, stream=None):
        """Autotune the segment size on this batch (dry runs).  Returns
        (best KiB, {candidate KiB: ms})."""
        reqs = np.ascontiguousarray(reqs)
        cand = CANDIDATES_KIB if candidates is None else list(candidates)
        ca = np.ascontiguousarray(cand, dtype=np.uint32)
        ms = np.zeros(len(cand), dtype=np.float32)
        best = u32(0)
        check(cg_tune_batch(self._h, reqs.ctypes.data, len(reqs), ca.ctypes.data, len(cand),
                            repeats, 1 if remember else 0, ms.ctypes.data, ctypes.byref(best),
                            _stream_handle(stream)), "cg_tune_batch")
        return int(best.value), {int(k): float(v) for k, v in zip(cand, ms)}

    def set_cost_model(self, weights: np.ndarray | None, hidden: int = 0) -> None:
        if weights is None:
            check(cg_set_cost_model(self._h, None, 0))
            return
        w = np.ascontiguousarray(weights, dtype=np.float32)
        check(cg_set_cost_model(self._h, w.ctypes.data, hidden), "cg_set_cost_model")

    def save_tuning(self, path: str) -> int:
        """Write the tuned split entries to a JSON file; returns how many."""
        import json
        n = u32(0)
        check(cg_get_tuned(self._h, None, None, 0, ctypes.byref(n)), "cg_get_tuned")
        k = n.value
        feat = np.zeros((max(1, k), NFEAT), dtype=np.float32)
        kib = np.zeros(max(1, k), dtype=np.uint32)
        check(cg_get_tuned(self._h, feat.ctypes.data, kib.ctypes.data, k, ctypes.byref(n)),
              "cg_get_tuned")
        with open(path, "w") as f:
            json.dump({"nfeat": NFEAT, "features": feat[:k].tolist(),
                       "segment_kib": kib[:k].tolist()}, f)
        return k

    def load_tuning(self, path: str) -> int:
        """Add the tuned split entries of a JSON file written by save_tuning."""
        import json
        d = json.load(open(path))
        if d["nfeat"] != NFEAT:
            raise ValueError(f"tuning file has {d['nfeat']} features, libcg uses {NFEAT}")
        feat = np.ascontiguousarray(d["features"], dtype=np.float32).reshape(-1, NFEAT)
        kib = np.ascontiguousarray(d["segment_kib"], dtype=np.uint32)
        check(cg_add_tuned(self._h, feat.ctypes.data, kib.ctypes.data, len(kib)), "cg_add_tuned")
        return len(kib)

    def choose_segment(self, reqs: np.ndarray) -> tuple[int, int]:
        reqs = np.ascontiguousarray(reqs)
        k, src = u32(0), u32(0)
        check(cg_choose_segment(self._h, reqs.ctypes.data, len(reqs), ctypes.byref(k),
                                ctypes.byref(src)))
        return int(k.value), int(src.value)

    # ------------------------------------------------------------ serving
    def serve_start(self, **cfg) -> None:
        c = cg_serve_config()
        for k, v in cfg.items():
            setattr(c, k, v)
        check(cg_serve_start(self._h, ctypes.byref(c)), "cg_serve_start")

    def submit(self, client: int, op: int, kind: int = 0, dst: int = 0, src: int = 0,
               n: int = 0) -> tuple[int, int]:
        t = u64(0)
        st = cg_submit(self._h, client, ctypes.byref(cg_request(op, kind, dst, src, n)),
                       ctypes.byref(t))
        return st, int(t.value)

    def wait(self, ticket: int, timeout_ms: int = 60000):
        r = cg_result()
        st = cg_wait(self._h, ticket, timeout_ms, ctypes.byref(r))
        return st, r

    def serve_replay(self, reqs: np.ndarray, clients: np.ndarray,
                     arrival_ns: np.ndarray) -> np.ndarray:
        """Replay a timed trace (REQUEST_DTYPE records); returns RESULT_DTYPE."""
        reqs = np.ascontiguousarray(reqs)
        assert reqs.dtype.itemsize == 32
        cl = np.ascontiguousarray(clients, dtype=np.uint32)
        ar = np.ascontiguousarray(arrival_ns, dtype=np.uint64)
        out = np.zeros(len(reqs), dtype=RESULT_DTYPE)
        check(cg_serve_replay(self._h, reqs.ctypes.data, cl.ctypes.data, ar.ctypes.data,
                              len(reqs), out.ctypes.data), "cg_serve_replay")
        return out

    def serve_stop(self) -> dict:
        s = cg_serve_stats()
        check(cg_serve_stop(self._h, ctypes.byref(s)), "cg_serve_stop")
        return {f: getattr(s, f) for f, _ in cg_serve_stats._fields_}

    def device_table(self, stream=None) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
        """(base, size, shadow) of the device copy of the allocation table."""
        n = u64(0)
        check(cg_device_table(self._h, None, None, None, 0, ctypes.byref(n),
                              _stream_handle(stream)), "cg_device_table")
        k = n.value
        out = [np.zeros(max(1, k), dtype=np.uint64) for _ in range(3)]
        check(cg_device_table(self._h, out[0].ctypes.data, out[1].ctypes.data, out[2].ctypes.data,
                              k, ctypes.byref(n), _stream_handle(stream)), "cg_device_table")
        return tuple(a[:k] for a in out)

    def stats(self) -> dict:
        s = cg_stats()
        check(cg_get_stats(self._h, ctypes.byref(s)))
        d = {f: getattr(s, f) for f, _ in cg_stats._fields_ if f != "errors"}
        d["errors"] = list(s.errors)
        return d


def plan_levels(reqs: np.ndarray, carry: bool = True,
                modes: np.ndarray | None = None) -> tuple[np.ndarray, int]:
    """Dependency levels of a batch (host only, see cg_plan_levels)."""
    reqs = np.ascontiguousarray(reqs)
    lv = np.zeros(len(reqs), dtype=np.int32)
    nl = u32(0)
    mp = None
    if modes is not None:
        modes = np.ascontiguousarray(modes, dtype=np.uint8)
        mp = modes.ctypes.data
    check(cg_plan_levels(reqs.ctypes.data if len(reqs) else None, len(reqs), int(carry), mp,
                         lv.ctypes.data if len(reqs) else None, ctypes.byref(nl)),
          "cg_plan_levels")
    return lv, int(nl.value)


def plan_units(reqs: np.ndarray, host_n: int, piece_rows: int, carry: bool = True,
               modes: np.ndarray | None = None) -> np.ndarray:
    """The batch planner's units (host only, see cg_plan_units): a structured
    array of (req, row_lo, row_hi, level) in request order."""
    reqs = np.ascontiguousarray(reqs)
    mp = None
    if modes is not None:
        modes = np.ascontiguousarray(modes, dtype=np.uint8)
        mp = modes.ctypes.data
    cap = len(reqs) + 1
    if piece_rows:
        cap += int((reqs["n"].astype(np.uint64) // np.uint64(512 * piece_rows)).sum()) + len(reqs)
    out = [np.zeros(cap, dtype=t) for t in (np.uint32, np.uint32, np.uint32, np.int32)]
    n = u64(0)
    check(cg_plan_units(reqs.ctypes.data if len(reqs) else None, len(reqs), int(carry), mp,
                        host_n, piece_rows, *[a.ctypes.data for a in out], cap, ctypes.byref(n)),
          "cg_plan_units")
    k = n.value
    res = np.zeros(k, dtype=[("req", "<u4"), ("row_lo", "<u4"), ("row_hi", "<u4"),
                             ("level", "<i4")])
    for f, a in zip(res.dtype.names, out):
        res[f] = a[:k]
    return res


CANDIDATES_KIB = [4, 8, 16, 32, 64, 128, 256, 512, 1024]
NFEAT = 13


def batch_features(reqs: np.ndarray) -> np.ndarray:
    reqs = np.ascontiguousarray(reqs)
    f = np.zeros(NFEAT, dtype=np.float32)
    check(cg_batch_features(reqs.ctypes.data if len(reqs) else None, len(reqs), f.ctypes.data))
    return f


def mlp_nweights(hidden: int) -> int:
    d = NFEAT + 1
    return 2 * d + d * hidden + 2 * hidden + 1


def mlp_fit(x: np.ndarray, t: np.ndarray, hidden: int = 32, epochs: int = 2000,
            lr: float = 3e-3, seed: int = 0) -> tuple[np.ndarray, np.ndarray]:
    """Train the cost model on the GPU; returns (weights, losses)."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    t = np.ascontiguousarray(t, dtype=np.float32)
    assert x.ndim == 2 and x.shape[1] == NFEAT + 1 and len(t) == len(x)
    w = np.zeros(mlp_nweights(hidden), dtype=np.float32)
    losses = np.zeros(epochs, dtype=np.float32)
    check(cg_mlp_fit(x.ctypes.data, t.ctypes.data, len(t), hidden, epochs, lr, seed,
                     w.ctypes.data, losses.ctypes.data, None), "cg_mlp_fit")
    return w, losses


def mlp_grad(x: np.ndarray, t: np.ndarray, weights: np.ndarray, hidden: int):
    x = np.ascontiguousarray(x, dtype=np.float32)
    t = np.ascontiguousarray(t, dtype=np.float32)
    w = np.ascontiguousarray(weights, dtype=np.float32)
    g = np.zeros_like(w)
    loss = ctypes.c_float(0)
    check(cg_mlp_grad(x.ctypes.data, t.ctypes.data, len(t), hidden, w.ctypes.data,
                      g.ctypes.data, ctypes.byref(loss), None), "cg_mlp_grad")
    return g, float(loss.value)


def format_report(rep: dict, kind: int) -> str:
    r = cg_report(**{k: rep[k] for k in REPORT_FIELDS})
    buf = ctypes.create_string_buffer(4096)
    check(cg_format_report(ctypes.byref(r), kind, buf, len(buf)))
    return buf.value.decode()

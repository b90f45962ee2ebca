"""Benchmark: single-transfer shadow checks (host->device scan + V carry) on
large synthetic transfers, through libcg's C ABI.

Workload (default): one host->device check each of 256 MiB, 1 GiB and
4 GiB from a 4 GiB host shadow image (V undefined density 1e-6 in sparse
runs, fully addressable) against a 16-entry allocation table.  One step =
the three checks.  Every input is larger than L2 (129 MB), so no flush is
needed between iterations.

Prints ONE JSON line (rank 0).  `--impl reference` times the CPU oracle on
a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import cg_synth as S  # noqa: E402

GB = 1e9
BYTES_PER_BYTE_CARRY = 2.125  # V read 1 + A read 1/8 + device V write 1
BYTES_PER_BYTE_SCAN = 1.125  # V read 1 + A read 1/8 (what crosses the host link)


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons while running.
    start() returns once the sampler has written its first sample, so the
    region that follows is covered; stop() keeps the samples taken between
    start() and stop() (by their timestamps), or the first one after start()
    when the region was shorter than one sampling interval."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.idx = device_index
        self.proc = None
        self.path = None

    def start(self):
        import shutil
        import tempfile
        if shutil.which("nvidia-smi") is None:
            return
        try:
            fd, self.path = tempfile.mkstemp(prefix=f"cg_clocks_{self.idx}_", suffix=".csv")
            self.f = os.fdopen(fd, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
            if self.path:
                self.f.close()
                os.unlink(self.path)
            return
        t_end = time.time() + 5.0
        while time.time() < t_end and self.proc.poll() is None:
            self.f.flush()
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.005)
        self.t0 = time.time()

    @staticmethod
    def _stamp(text: str) -> float | None:
        import datetime
        for fmt in ("%Y/%m/%d %H:%M:%S.%f", "%Y/%m/%d %H:%M:%S"):
            try:
                return datetime.datetime.strptime(text, fmt).timestamp()
            except ValueError:
                continue
        return None

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        t1 = time.time()
        time.sleep(0.05)  # one more sample past the region's end
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        rows = []
        with open(self.path) as fh:
            lines = fh.read().splitlines()
        os.unlink(self.path)
        for line in lines:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                rows.append((self._stamp(parts[0]), float(parts[2]), float(parts[3]), parts[6:10]))
            except ValueError:
                continue
        if not rows:
            return None
        inside = [r for r in rows if r[0] is not None and self.t0 <= r[0] <= t1]
        if not inside:
            after = [r for r in rows if r[0] is not None and r[0] >= self.t0]
            inside = after[:1] or rows[-1:]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, _, r in inside for i, x in enumerate(r)
                          if x == "Active"})
        return {"sm_mhz": statistics.median(r[1] for r in inside), "sm_max_mhz": inside[0][2],
                "reasons": reasons, "samples": len(inside),
                "region_s": round(t1 - self.t0, 3)}


def reduce_max(value: float, device=None) -> float:
    """The largest of `value` over all ranks (the job's time is its slowest
    rank's); the value itself when not distributed."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate(bytes_per_rank: int, elapsed_ms_per_rank: float, device=None) -> tuple[float, float]:
    """Whole-job throughput (GB/s) from every rank's own work and time:
    all ranks' bytes over the slowest rank's time."""
    import torch.distributed as dist
    world = dist.get_world_size() if dist.is_available() and dist.is_initialized() else 1
    ms = reduce_max(elapsed_ms_per_rank, device)
    return bytes_per_rank * world / (ms / 1e3) / GB, ms


def build_workload(sizes):
    w = S.large(0, sizes=sizes)
    return w


def run_cg(args, world, rank, local):
    import torch

    import paper_1310_0901_gb300 as cg

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    sizes = tuple(int(x) << 20 for x in args.sizes_mib.split(","))
    w = build_workload(sizes)
    n_img = w.image.n
    a_host = torch.from_numpy(w.image.a_bits[: n_img // 8].copy()).pin_memory()
    v_host = torch.from_numpy(w.image.v).pin_memory()
    a_dev = a_host.to(dev)
    v_dev = v_host.to(dev)
    ctx = cg.Context(scan_engine=args.engine)
    ctx.bind_host_shadow(a_dev, v_dev)
    order = np.argsort(w.table.base)
    for b, s in zip(w.table.base[order], w.table.size[order]):
        cg.check(ctx.register_alloc(int(b), int(s)), "register")
    reqs = [cg.cg_copy(int(q["kind"]), 0, int(q["dst"]), int(q["src"]), int(q["n"]))
            for q in w.reqs]
    bytes_per_step = sum(int(q["n"]) for q in w.reqs)
    stream = torch.cuda.current_stream(dev)
    sh = stream.cuda_stream
    rep_dev = torch.zeros((len(reqs), cg.REPORT_DTYPE.itemsize), dtype=torch.uint8, device=dev)
    import ctypes

    def step_async(events=None):
        for i, q in enumerate(reqs):
            if events is not None:
                events[i][0].record(stream)
            cg.check(cg.cg_check_copy_async(ctx.handle, ctypes.byref(q),
                                            rep_dev[i].data_ptr(), sh), "check_async")
            if events is not None:
                events[i][1].record(stream)

    # warm-up (also validates the reports once against expectations)
    for _ in range(args.warmup):
        step_async()
    torch.cuda.synchronize()
    reps = np.frombuffer(rep_dev.cpu().numpy().tobytes(), dtype=cg.REPORT_DTYPE)
    planted = np.zeros(n_img, bool)
    for s0, ln in w.image.undef_runs:
        planted[s0:s0 + ln] = True
    for i, q in enumerate(w.reqs):
        n = int(q["n"])
        assert int(reps[i]["n_undef"]) == int(planted[:n].sum()), "report mismatch"
        assert int(reps[i]["flags"]) in (0, cg.FLAGS["HOST_UNDEF"])

    clocks = Clocks(local)
    clocks.start()
    # the clock record covers the timed region and, just before it, about
    # half a second of the same untimed steps (the timed region alone is a
    # few tens of milliseconds at the default step count)
    s_env = time.perf_counter()
    while time.perf_counter() - s_env < 0.5:
        step_async()
        torch.cuda.synchronize()
    k0 = ctx.stats()["kernels"]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    t_region = time.time()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    ev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in reqs] for _ in range(args.steps)]
    t0.record(stream)
    for k in range(args.steps):
        step_async(ev[k])
    t1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    if clk is not None:
        clk["timed_region_s"] = round(time.time() - t_region, 3)
        clk["window"] = "the timed region and the 0.5 s of identical untimed steps before it"
    launches = ctx.stats()["kernels"] - k0
    elapsed_ms = t0.elapsed_time(t1)
    # per-kernel durations (the scan kernel is the only launch per check)
    kern_ms = np.array([[ev[k][i][0].elapsed_time(ev[k][i][1]) for i in range(len(reqs))]
                        for k in range(args.steps)])
    value, elapsed_ms = aggregate(bytes_per_step * args.steps, elapsed_ms, dev)

    # roofline of the dominant kernel: the largest transfer's scan+carry
    big = int(np.argmax([int(q["n"]) for q in w.reqs]))
    kmean = float(kern_ms[:, big].mean())
    alg_bytes = BYTES_PER_BYTE_CARRY * int(w.reqs[big]["n"])
    achieved = alg_bytes / (kmean / 1e3) / GB
    peak, peak_kind = _peaks()
    traffic = _profiled_traffic() if args.engine != 1 and sizes == LARGE_DEFAULT else None

    # end to end through the C ABI: per step upload each transfer's host
    # shadow (V + A) from pinned host memory, check, read the report
    e2e_ms = None
    h2d = 0
    d2h = 0
    if args.e2e_steps > 0:
        for q in w.reqs:  # one untimed step (first use of the pinned image by the copy engines)
            n = int(q["n"])
            ctx.upload_host_shadow(a_host, v_host, int(q["src"]), n, stream)
            cg.check(ctx.check_copy(int(q["kind"]), int(q["dst"]), int(q["src"]), n, stream)[0],
                     "check_copy")
        torch.cuda.synchronize()
        s0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            for q in w.reqs:
                n = int(q["n"])
                ctx.upload_host_shadow(a_host, v_host, int(q["src"]), n, stream)
                st, rep = ctx.check_copy(int(q["kind"]), int(q["dst"]), int(q["src"]), n, stream)
                cg.check(st, "check_copy")
        torch.cuda.synchronize()
        e2e_ms = (time.perf_counter() - s0) * 1e3
        h2d = int(sum(int(q["n"]) + int(q["n"]) // 8 for q in w.reqs))
        d2h = cg.REPORT_DTYPE.itemsize * len(reqs)
    if e2e_ms is not None:
        e2e_ms = reduce_max(e2e_ms, dev)
    # end to end, in place: the kernel reads the pinned host shadow over the
    # host link (no staging copy); the carry still lands in HBM
    zc_ms = None
    if args.e2e_steps > 0:
        ctx_h = cg.Context()
        ctx_h.bind_host_shadow(a_host, v_host)
        for b, s_ in zip(w.table.base[order], w.table.size[order]):
            cg.check(ctx_h.register_alloc(int(b), int(s_)), "register")
        for q in w.reqs:  # untimed pass (first-touch of the device shadow)
            cg.check(ctx_h.check_copy(int(q["kind"]), int(q["dst"]), int(q["src"]), int(q["n"]),
                                      stream)[0], "check_copy")
        torch.cuda.synchronize()
        s0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            for i, q in enumerate(w.reqs):
                st, rep = ctx_h.check_copy(int(q["kind"]), int(q["dst"]), int(q["src"]),
                                           int(q["n"]), stream)
                cg.check(st, "check_copy")
                assert rep["n_undef"] == int(reps[i]["n_undef"])
        torch.cuda.synchronize()
        zc_ms = reduce_max((time.perf_counter() - s0) * 1e3, dev)
        ctx_h.close()

    out = {
        "metric": "shadow GB/s checked vs HBM peak (single large host->device transfer checks)",
        "value": round(value, 2),
        "unit": "GB/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(elapsed_ms / args.steps, 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u8",
        "data": "synthetic (seeded cg_synth.large: V undefined density 1e-6 in runs, A all addressable)",
        "config": {"workload": w.name, "checks_per_step": len(reqs),
                   "bytes_checked_per_step": bytes_per_step,
                   "l2": "inputs larger than L2 (each transfer >= 256 MiB); no flush",
                   "parallelism": f"replicas x{world}", "carry": True},
        "roofline": {"bound": "hbm",
                     "kernel": ("scan_single_kernel<HTOD,carry>" if args.engine == 1
                                else "scan_single_tma_kernel<HTOD,carry>"),
                     "bytes_per_checked_byte": BYTES_PER_BYTE_CARRY,
                     "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "peak_source": peak_kind,
                     "traffic": traffic, "kernel_ms_mean": round(kmean, 4),
                     "kernel_ms_per_size": {f"{int(q['n']) >> 20}MiB":
                                            round(float(kern_ms[:, i].mean()), 4)
                                            for i, q in enumerate(w.reqs)}},
        "gpu_launches": int(launches),
    }
    # the copy engines' rate for a plain pinned host->device copy (1 GiB of
    # the image copied onto itself), for context: the in-place mode reads
    # the host image with kernel loads over the host link instead
    link_gbs = None
    if args.e2e_steps > 0:
        m = min(1 << 30, n_img)
        for _ in range(2):
            v_dev[:m].copy_(v_host[:m], non_blocking=True)
        c0 = torch.cuda.Event(enable_timing=True)
        c1 = torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        for _ in range(4):
            v_dev[:m].copy_(v_host[:m], non_blocking=True)
        c1.record(stream)
        torch.cuda.synchronize()
        link_gbs = 4 * m / (c0.elapsed_time(c1) / 1e3) / GB
    if e2e_ms is not None:
        up = bytes_per_step * args.e2e_steps * world / (e2e_ms / 1e3) / GB
        inplace = bytes_per_step * args.e2e_steps * world / (zc_ms / 1e3) / GB if zc_ms else 0.0
        # two records, one per way a caller holds the host image in pinned
        # host memory; each counts the host->device bytes of its own step
        # (a check needs 1.125 B of host shadow, V + A, per checked byte)
        out["e2e"] = {"value": round(inplace, 2), "unit": "GB/s",
                      "mode": "in place: cg_check_copy on the pinned host image bound with "
                              "cg_bind_host_shadow; the kernels read V and A over the host link",
                      "h2d_bytes_per_step": h2d, "h2d_by": "kernel loads over NVLink-C2C",
                      "d2h_bytes_per_step": d2h, "steps": args.e2e_steps,
                      "host_read_gbs": round(inplace * BYTES_PER_BYTE_SCAN, 1)}
        out["e2e_upload_then_check"] = {
            "value": round(up, 2), "unit": "GB/s",
            "mode": "cg_upload_host_shadow (copy engine, pinned host -> HBM) then "
                    "cg_check_copy, per transfer",
            "h2d_bytes_per_step": h2d, "h2d_by": "cudaMemcpyAsync",
            "d2h_bytes_per_step": d2h, "steps": args.e2e_steps}
        if link_gbs:
            out["e2e_upload_then_check"]["host_copy_gbs"] = round(link_gbs, 1)
    if clk is not None:
        out["clocks"] = clk
    ctx.close()
    return out, w


LARGE_DEFAULT = (256 << 20, 1 << 30, 4 << 30)


def run_batched_workload(args, which: str):
    """Batched checks (one cg_check_batch per step) against one synchronous
    cg_check_copy per copy, on the same GPU and workload."""
    import torch

    import paper_1310_0901_gb300 as cg
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    t_gen = time.perf_counter()
    w = S.batched(0) if which == "batched" else S.adversarial(0)
    t_gen = time.perf_counter() - t_gen
    n_img = w.image.n
    a_dev = torch.from_numpy(w.image.a_bits[: n_img // 8].copy()).to(dev)
    v_dev = torch.from_numpy(w.image.v).to(dev)
    ctx = cg.Context(batch_segment_kib=args.segment_kib, batch_autotune=1,
                     batch_piece_kib=args.piece_kib)
    ctx.bind_host_shadow(a_dev, v_dev)
    order = np.argsort(w.table.base)
    t_reg = time.perf_counter()
    st = ctx.register_allocs(w.table.base[order], w.table.size[order])
    assert not st.any()
    t_reg = time.perf_counter() - t_reg
    reqs = w.reqs
    nreq = len(reqs)
    bytes_per_batch = int(reqs["n"].sum())
    stream = torch.cuda.current_stream(dev)
    reps_out = np.empty(nreq, dtype=cg.REPORT_DTYPE)   # result buffers reused across batches
    recs_out = np.empty(8 * nreq, dtype=cg.RECORD_DTYPE)
    # the split is autotuned online: the warm-up batches try the candidates
    # (real runs, timed), the timed batches use the fastest
    for _ in range(max(args.warmup, 5 if not args.segment_kib else 0)):
        stt, reps, recs, total, _ = ctx.check_batch(reqs, 8 * nreq, None, reps_out, recs_out)
        cg.check(stt, "check_batch")
    s0 = ctx.stats()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        stt, reps, recs, total, _ = ctx.check_batch(reqs, 8 * nreq, None, reps_out, recs_out)
        cg.check(stt, "check_batch")
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    s1 = ctx.stats()
    # pipelined: two batches in flight, the next one looked up and planned on
    # the host while the one before runs (cg_check_batch_async)
    reps = reps.copy()  # the last synchronous batch's reports (the roofline reads them)
    host_s = {"submit": 0.0, "wait": 0.0}

    def pipelined(k):
        pend = []
        for _ in range(k):
            h0 = time.perf_counter()
            stt, t, _ = ctx.check_batch_async(reqs, rec_cap=8 * nreq)
            host_s["submit"] += time.perf_counter() - h0
            cg.check(stt, "check_batch_async")
            pend.append(t)
            if len(pend) == 2:
                h0 = time.perf_counter()
                cg.check(ctx.batch_wait(pend.pop(0), nreq, 8 * nreq, reps_out, recs_out)[0],
                         "batch_wait")
                host_s["wait"] += time.perf_counter() - h0
        for t in pend:
            h0 = time.perf_counter()
            cg.check(ctx.batch_wait(t, nreq, 8 * nreq, reps_out, recs_out)[0], "batch_wait")
            host_s["wait"] += time.perf_counter() - h0
    pipelined(2)
    torch.cuda.synchronize()
    host_s["submit"] = host_s["wait"] = 0.0
    sp0 = ctx.stats()
    tp = time.perf_counter()
    pipelined(args.steps)
    torch.cuda.synchronize()
    dt_pipe = time.perf_counter() - tp
    sp1 = ctx.stats()
    host_s["of_which_lookup"] = (sp1["batch_lookup_ns"] - sp0["batch_lookup_ns"]) / 1e9
    host_s["of_which_plan"] = (sp1["batch_plan_ns"] - sp0["batch_plan_ns"]) / 1e9
    levels = (s1["levels"] - s0["levels"]) / args.steps
    launches = (s1["kernels"] - s0["kernels"]) / args.steps
    per_batch_ms = {k: round((s1[k] - s0[k]) / args.steps / 1e6, 2)
                    for k in ("batch_ns", "batch_plan_ns", "batch_lookup_ns")}
    # one launch per copy: every copy of the same stream, one cg_check_copy each
    m = min(nreq, args.single_sample)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    for q in reqs[:m]:
        stt, _ = ctx.check_copy(int(q["kind"]), int(q["dst"]), int(q["src"]), int(q["n"]), stream)
        cg.check(stt, "check_copy")
    torch.cuda.synchronize()
    dt1 = time.perf_counter() - t1
    sync_cps = nreq * args.steps / dt
    batch_cps = nreq * args.steps / dt_pipe
    single_cps = m / dt1
    # algorithmic HBM bytes of one batch, from its verdicts: the host scan
    # always runs (V + A of host bytes), device V is read only from a valid
    # source and written only when every device range is valid
    f = reps["flags"].astype(np.int64)
    n = reqs["n"].astype(np.float64)
    kind = reqs["kind"]
    dst_ok = (f & (cg.FLAGS["UNALLOC_DST"] | cg.FLAGS["OVERRUN_DST"])) == 0
    src_ok = (f & (cg.FLAGS["UNALLOC_SRC"] | cg.FLAGS["OVERRUN_SRC"])) == 0
    alg = np.where(kind == S.HTOD, 1.125 * n + n * dst_ok,
                   np.where(kind == S.DTOH, 0.125 * n + 2 * n * src_ok,
                            n * src_ok + n * (src_ok & dst_ok)))
    alg_bytes = float(alg.sum())
    peak, peak_kind = _peaks()
    gpu_ms = per_batch_ms["batch_ns"] - per_batch_ms["batch_plan_ns"] - per_batch_ms["batch_lookup_ns"]
    roof = {"bound": "hbm", "algorithmic_bytes_per_batch": int(alg_bytes),
            "achieved": round(alg_bytes / (dt_pipe / args.steps) / GB, 1), "peak": peak,
            "unit": "GB/s",
            "frac": round(alg_bytes / (dt_pipe / args.steps) / GB / peak, 4),
            "frac_one_batch_at_a_time": round(alg_bytes / (dt / args.steps) / GB / peak, 4),
            "frac_during_level_kernels": round(alg_bytes / (gpu_ms / 1e3) / GB / peak, 4)
            if gpu_ms > 0 else None,
            "peak_source": peak_kind}
    out = {
        "metric": "batched checks/sec",
        "value": round(batch_cps, 1), "unit": "checks/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(dt_pipe / args.steps * 1e3, 3),
        "mode": "two batches in flight (cg_check_batch_async)",
        "host_ms_per_batch": {k: round(v / args.steps * 1e3, 2) for k, v in host_s.items()},
        "one_batch_at_a_time": {"checks_per_s": round(sync_cps, 1),
                                "ms_per_batch": round(dt / args.steps * 1e3, 3)},
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic (seeded cg_synth." + which + ")",
        "config": {"workload": w.name, "requests": nreq, "allocations": int(len(w.table.base)),
                   "bytes_checked_per_batch": bytes_per_batch,
                   "levels_per_batch": levels,
                   "l2": "working set larger than L2", "carry": True},
        "batched_gb_per_s": round(bytes_per_batch * args.steps / dt_pipe / GB, 1),
        "roofline": roof,
        "one_launch_per_copy": {"checks_per_s": round(single_cps, 1), "sample": m,
                                "gb_per_s": round(int(reqs["n"][:m].sum()) / dt1 / GB, 1)},
        "speedup_vs_one_launch_per_copy": round(batch_cps / single_cps, 2),
        "records_per_batch": int(total),
        "split": {"segment_kib": ctx.choose_segment(reqs)[0],
                  "source": ["default", "autotuned", "learned", "fixed", "trial"][
                      ctx.choose_segment(reqs)[1]]},
        "batch_breakdown_ms": {"total": per_batch_ms["batch_ns"],
                               "host_plan": per_batch_ms["batch_plan_ns"],
                               "lookup_and_readback": per_batch_ms["batch_lookup_ns"]},
        "gpu_launches": launches,
        "setup_s": {"generate": round(t_gen, 1), "register": round(t_reg, 1)},
        "records_per_s": round(total * args.steps / dt_pipe, 1),
    }
    ctx.close()
    del a_dev, v_dev
    torch.cuda.empty_cache()
    if args.cpu_budget_s > 0:
        out.update(oracle_copy_baselines(w.image, w.table, reqs, args.cpu_budget_s, which))
    return out


def _serving_image(host_n: int):
    """The serving workload's host image on the host: V (zero but for the
    planted undefined runs) and the positions the runs cover."""
    vh = np.zeros(host_n, np.uint8)
    starts, lengths, values = S.serving_image_runs(0, host_n)
    for s0, ln, val in zip(starts, lengths, values):
        vh[s0:s0 + ln] = val
    idx = np.unique(np.concatenate([np.arange(s0, s0 + ln) for s0, ln in zip(starts, lengths)]))
    return vh, idx


def _serve_context(cg, torch, dev, tr, v, a):
    ctx = cg.Context()
    ctx.bind_host_shadow(a, v)
    order = np.argsort(tr.table.base)
    assert not ctx.register_allocs(tr.table.base[order], tr.table.size[order]).any()
    return ctx


def _latency(res, tr):
    checks = tr.reqs["op"] == S.OP_CHECK
    lat_us = (res["done_ns"][checks] - res["submit_ns"][checks]).astype(np.float64) / 1e3
    span_s = (int(res["done_ns"].max()) - int(res["submit_ns"].min())) / 1e9
    return lat_us, span_s, int(checks.sum())


def oracle_serving_baseline(tr, host_n: int, budget_s: float) -> dict:
    """The oracle, as it stands, replaying the serving trace on one host
    core: requests in arrival order, each applied to one oracle state (the
    32 GiB image and the allocation table) as soon as the previous one is
    done.  Each request's service time is measured; its latency is the
    time from its arrival to the end of its service in that single queue.
    Bounded: the requests that fit in the budget.  One thread: a state per
    thread would need its own 36 GiB image copy."""
    import oracle as O
    vh, _ = _serving_image(host_n)
    orc = O.Oracle(np.full(host_n // 8, 0xFF, np.uint8), vh)
    del vh
    order = np.argsort(tr.table.base)
    assert not orc.register_allocs(tr.table.base[order], tr.table.size[order]).any()
    svc = []
    t = 0.0
    for q in tr.reqs:
        op = int(q["op"])
        s0 = time.perf_counter()
        if op == S.OP_CHECK:
            orc.check_copy_status(int(q["kind"]), int(q["dst"]), int(q["src"]), int(q["n"]))
        elif op == S.OP_ALLOC:
            orc.register_alloc(int(q["dst"]), int(q["n"]))
        elif op == S.OP_FREE:
            orc.free(int(q["dst"]))
        else:
            orc.mark(int(q["dst"]), int(q["n"]), 0 if op == S.OP_MARK_DEFINED else 0xFF)
        dt = time.perf_counter() - s0
        svc.append(dt)
        t += dt
        if t >= budget_s:
            break
    orc.close()
    m = len(svc)
    arr = tr.arrival_ns[:m].astype(np.float64) / 1e9
    done = np.empty(m)
    free_at = 0.0
    for i in range(m):
        free_at = max(arr[i], free_at) + svc[i]
        done[i] = free_at
    checks = tr.reqs["op"][:m] == S.OP_CHECK
    lat_us = (done - arr)[checks] * 1e6
    return {"value": round(int(checks.sum()) / t, 1), "unit": "checks/s", "cores": 1,
            "kind": "oracle", "cpu": _cpu_model(),
            "latency_us": {"p50": round(float(np.percentile(lat_us, 50)), 1),
                           "p99": round(float(np.percentile(lat_us, 99)), 1)},
            "sample": f"the first {m} requests of the trace ({arrival_span(tr, m):.3f} s of "
                      f"arrivals) replayed in arrival order through one oracle state, 1 thread, "
                      f"{t:.1f} s of service"}


def arrival_span(tr, m):
    return (int(tr.arrival_ns[m - 1]) - int(tr.arrival_ns[0])) / 1e9 if m > 1 else 0.0


SERVE_CFG = dict(clients=8, ring_capacity=1 << 14, max_round=8192, budget_bytes=8 << 30)
SWEEP_RATES = (400_000.0, 800_000.0, 1_600_000.0, 3_200_000.0)
SWEEP_SECONDS = 1.0
SWEEP_P99_BOUND_US = 1000.0


def run_serving(args):
    """The serving loop under Poisson arrivals from 8 client threads:
    sustained checks/s and submit-to-result latency percentiles; the same
    engine at higher offered rates; one synchronous cg_check_copy per
    request on the same size mix; the oracle replaying the trace."""
    import torch

    import paper_1310_0901_gb300 as cg
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    host_n = args.serve_image_gib << 30
    tr = S.serving(0, seconds=args.serve_seconds, rate=args.serve_rate, host_n=host_n)
    vh, idx = _serving_image(host_n)
    v = torch.zeros(host_n, dtype=torch.uint8, device=dev)
    a = torch.full((host_n // 8,), 0xFF, dtype=torch.uint8, device=dev)
    idx_d = torch.from_numpy(idx).to(dev)
    vals_d = torch.from_numpy(vh[idx]).to(dev)
    del vh

    def reset_image():  # each context below starts from the same image
        v.zero_()
        v[idx_d] = vals_d

    reset_image()
    ctx = _serve_context(cg, torch, dev, tr, v, a)
    cfg = dict(SERVE_CFG, streams=args.serve_streams)
    ctx.serve_start(**cfg)
    # warm-up: a short checks-only trace (no allocation events)
    wt = S.serve_trace(S.rng_for(99), 20_000, args.serve_rate, 8, tr.table, host_n,
                       event_frac=0.0)
    ctx.serve_replay(wt.reqs, wt.client, wt.arrival_ns)
    clocks = Clocks(0)
    clocks.start()
    res = ctx.serve_replay(tr.reqs, tr.client, tr.arrival_ns)
    clk = clocks.stop()
    stats = ctx.serve_stop()
    ctx.close()
    ok = res["status"] == 0
    lat_us, span_s, n_checks = _latency(res, tr)
    pct = {f"p{p}": round(float(np.percentile(lat_us, p)), 1) for p in (50, 90, 99, 99.9)}
    pct["max"] = round(float(lat_us.max()), 1)
    checks = tr.reqs["op"] == S.OP_CHECK
    sizes = tr.reqs["n"][checks]
    small = sizes <= 4096
    # offered-rate sweep: the same engine and configuration on a fresh
    # context per rate
    n_big = 100
    big = np.arange(len(tr.table.base) - n_big, len(tr.table.base))
    sweep = []
    for rate in SWEEP_RATES:
        reset_image()
        ts = S.serve_trace(S.rng_for(int(rate)), int(SWEEP_SECONDS * rate), rate, 8, tr.table,
                           host_n, big=big)
        c2 = _serve_context(cg, torch, dev, tr, v, a)
        c2.serve_start(**cfg)
        c2.serve_replay(wt.reqs, wt.client, wt.arrival_ns)
        r2 = c2.serve_replay(ts.reqs, ts.client, ts.arrival_ns)
        c2.serve_stop()
        c2.close()
        l2, sp2, nc2 = _latency(r2, ts)
        sweep.append({"offered_req_per_s": rate,
                      "offered_checks_per_s": round(nc2 / arrival_span(ts, len(ts.reqs)), 1),
                      "checks_per_s": round(nc2 / sp2, 1),
                      "p50_us": round(float(np.percentile(l2, 50)), 1),
                      "p99_us": round(float(np.percentile(l2, 99)), 1),
                      "all_ok": bool((r2["status"] == 0).all())})
    main_pt = {"offered_req_per_s": args.serve_rate,
               "offered_checks_per_s": round(n_checks / arrival_span(tr, len(tr.reqs)), 1),
               "checks_per_s": round(n_checks / span_s, 1), "p50_us": pct["p50"],
               "p99_us": pct["p99"], "all_ok": bool(ok.all())}
    pts = [main_pt] + sweep
    keeps_up = [p for p in pts if p["checks_per_s"] >= 0.95 * p["offered_checks_per_s"]
                and p["p99_us"] <= SWEEP_P99_BOUND_US]
    best = max(keeps_up, key=lambda p: p["checks_per_s"]) if keeps_up else None
    # one synchronous cg_check_copy per request on the same size mix
    reset_image()
    c3 = _serve_context(cg, torch, dev, tr, v, a)
    one = S.serve_trace(S.rng_for(7), 20_000, args.serve_rate, 8, tr.table, host_n, big=big,
                        event_frac=0.0)
    stream = torch.cuda.current_stream(dev)
    for q in one.reqs[:200]:
        cg.check(c3.check_copy(int(q["kind"]), int(q["dst"]), int(q["src"]), int(q["n"]),
                               stream)[0], "check_copy")
    torch.cuda.synchronize()
    lat1 = []
    t1 = time.perf_counter()
    for q in one.reqs:
        s0 = time.perf_counter()
        cg.check(c3.check_copy(int(q["kind"]), int(q["dst"]), int(q["src"]), int(q["n"]),
                               stream)[0], "check_copy")
        lat1.append((time.perf_counter() - s0) * 1e6)
    dt1 = time.perf_counter() - t1
    c3.close()
    del v, a, idx_d, vals_d
    torch.cuda.empty_cache()
    out = {
        "metric": "sustained checks/sec and p50/p99 check latency (serving)",
        "value": round(n_checks / span_s, 1), "unit": "checks/s", "n_gpus": 1,
        "higher_is_better": True, "dtype": "u8", "data": "synthetic (seeded cg_synth.serving)",
        "config": {"workload": tr.note, "requests": int(len(tr.reqs)), "checks": n_checks,
                   "offered_rate_per_s": args.serve_rate, "clients": 8,
                   "allocations": int(len(tr.table.base)), "host_image_bytes": host_n,
                   "serve_config": cfg},
        "latency_us": pct,
        "latency_us_checks_le_4KiB": {f"p{p}": round(float(np.percentile(lat_us[small], p)), 1)
                                      for p in (50, 99)},
        "all_ok": bool(ok.all()), "span_s": round(span_s, 3),
        "concurrent_access_findings": int(((res["report"]["flags"] & (1 << 8)) != 0).sum()),
        "offered_gb_per_s": round(float(sizes.sum()) / (args.serve_seconds * 1e9), 1),
        "serve_stats": stats,
        "rate_sweep": {"points": pts, "p99_bound_us": SWEEP_P99_BOUND_US,
                       "highest_sustained": best,
                       "note": f"{SWEEP_SECONDS:g} s of arrivals per higher rate, a fresh context each; a point "
                               "keeps up when it serves >= 95 % of the offered checks/s with "
                               "p99 within the bound"},
        "one_launch_per_copy": {
            "checks_per_s": round(len(one.reqs) / dt1, 1),
            "latency_us": {"p50": round(float(np.percentile(lat1, 50)), 1),
                           "p99": round(float(np.percentile(lat1, 99)), 1)},
            "sample": f"{len(one.reqs)} checks of the serving size mix, one synchronous "
                      "cg_check_copy each, one thread"},
    }
    if best:
        out["speedup_vs_one_launch_per_copy"] = round(best["checks_per_s"] / (len(one.reqs) / dt1), 2)
    if clk is not None:
        out["clocks"] = clk
    if args.cpu_budget_s > 0:
        out["cpu_baseline"] = oracle_serving_baseline(tr, host_n, args.cpu_budget_s)
        out["cpu_baseline_all_cores"] = {
            "value": None, "cores": _host_cores(),
            "why": "each thread would need its own oracle state holding the 32 GiB image "
                   "(36 GiB with the A bits); the host has less memory than that times the cores"}
    return out


def run_small(args):
    """The small correctness workload as a timed line: its 1,000 requests
    (1 B-16 KiB; overruns, freed targets, wild pointers) as one batch, two
    batches in flight, one synchronous cg_check_copy per request, and the
    oracle (one batch per pass, one thread; a state per thread on all
    cores)."""
    import threading

    import torch

    import paper_1310_0901_gb300 as cg
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    w = S.small(0)
    n_img = w.image.n
    a_dev = torch.from_numpy(w.image.a_bits[: n_img // 8].copy()).to(dev)
    v_dev = torch.from_numpy(w.image.v.copy()).to(dev)
    ctx = cg.Context()
    ctx.bind_host_shadow(a_dev, v_dev)
    order = np.argsort(w.table.base)
    assert not ctx.register_allocs(w.table.base[order], w.table.size[order]).any()
    for j in w.table.freed:
        ctx.free(int(w.table.base[j]))
    reqs = w.reqs
    nreq = len(reqs)
    reps_out = np.empty(nreq, dtype=cg.REPORT_DTYPE)
    recs_out = np.empty(8 * nreq, dtype=cg.RECORD_DTYPE)
    steps = max(args.steps, 20)
    for _ in range(max(args.warmup, 3)):
        cg.check(ctx.check_batch(reqs, 8 * nreq, None, reps_out, recs_out)[0], "check_batch")
    k0 = ctx.stats()["kernels"]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        stt, _, _, total, _ = ctx.check_batch(reqs, 8 * nreq, None, reps_out, recs_out)
        cg.check(stt, "check_batch")
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    launches = (ctx.stats()["kernels"] - k0) / steps
    pend = []
    torch.cuda.synchronize()
    tp = time.perf_counter()
    for _ in range(steps):
        stt, t, _ = ctx.check_batch_async(reqs, rec_cap=8 * nreq)
        cg.check(stt, "check_batch_async")
        pend.append(t)
        if len(pend) == 2:
            cg.check(ctx.batch_wait(pend.pop(0), nreq, 8 * nreq, reps_out, recs_out)[0], "wait")
    for t in pend:
        cg.check(ctx.batch_wait(t, nreq, 8 * nreq, reps_out, recs_out)[0], "wait")
    torch.cuda.synchronize()
    dtp = time.perf_counter() - tp
    stream = torch.cuda.current_stream(dev)
    t1 = time.perf_counter()
    for q in reqs:
        cg.check(ctx.check_copy(int(q["kind"]), int(q["dst"]), int(q["src"]), int(q["n"]),
                                stream)[0], "check_copy")
    torch.cuda.synchronize()
    dt1 = time.perf_counter() - t1
    ctx.close()
    del a_dev, v_dev
    torch.cuda.empty_cache()
    out = {
        "metric": "batched checks/sec (small workload)",
        "value": round(nreq * steps / dtp, 1), "unit": "checks/s", "n_gpus": 1, "steps": steps,
        "warmup": max(args.warmup, 3), "ms_per_step": round(dtp / steps * 1e3, 4),
        "mode": "two batches in flight (cg_check_batch_async)",
        "higher_is_better": True, "dtype": "u8", "data": "synthetic (seeded cg_synth.small)",
        "config": {"workload": "small-1000-req-64-live-allocs-1MiB-image", "requests": nreq,
                   "bytes_checked_per_batch": int(reqs["n"].sum())},
        "one_batch_at_a_time": {"checks_per_s": round(nreq * steps / dt, 1),
                                "ms_per_batch": round(dt / steps * 1e3, 4)},
        "one_launch_per_copy": {"checks_per_s": round(nreq / dt1, 1)},
        "speedup_vs_one_launch_per_copy": round((nreq * steps / dtp) / (nreq / dt1), 2),
        "records_per_batch": int(total), "gpu_launches_per_batch": launches,
    }
    if args.cpu_budget_s > 0:
        budget = min(args.cpu_budget_s, 5.0)
        orc = _oracle_state(w.image, w.table)
        run = orc.batch_runner(reqs)
        done = 0
        t = 0.0
        while t < budget:
            s0 = time.perf_counter()
            assert run() == 0
            t += time.perf_counter() - s0
            done += 1
        orc.close()
        out["cpu_baseline"] = {"value": round(done * nreq / t, 1), "unit": "checks/s",
                               "cores": 1, "kind": "oracle", "cpu": _cpu_model(),
                               "sample": f"{done} passes of the 1,000-request batch, 1 thread, "
                                         f"{t:.1f} s"}
        cores = _host_cores()
        states = [_oracle_state(w.image, w.table) for _ in range(cores)]
        runs = [o.batch_runner(reqs) for o in states]
        cnt = [0] * cores
        spent = [0.0] * cores
        start = threading.Barrier(cores + 1)

        def work(k):
            start.wait()
            s0 = time.perf_counter()
            while time.perf_counter() - s0 < budget / 2:
                assert runs[k]() == 0
                cnt[k] += 1
            spent[k] = time.perf_counter() - s0

        pool = [threading.Thread(target=work, args=(k,)) for k in range(cores)]
        for th in pool:
            th.start()
        start.wait()
        for th in pool:
            th.join()
        for o in states:
            o.close()
        out["cpu_baseline_all_cores"] = {
            "value": round(sum(cnt) * nreq / max(spent), 1), "unit": "checks/s", "cores": cores,
            "kind": "oracle", "cpu": _cpu_model(),
            "sample": f"{sum(cnt)} passes of the batch over {cores} threads, each with its own "
                      f"oracle state, {max(spent):.1f} s"}
    return out


def run_pitched(args):
    """Full-size pitched host->device checks with carry (cg_check_copy3d_async,
    one launch each): 256 MiB of 16 KiB rows at a 16.5 KiB pitch, and a
    16-byte field of 16M 24-byte records (the strided host read of the
    paper's footnote).  Kernel time by CUDA events around the back-to-back
    launches of the timed region (and, for comparison, around each launch)."""
    import ctypes

    import torch

    import paper_1310_0901_gb300 as cg

    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream(dev)
    sh = stream.cuda_stream
    peak, peak_kind = _peaks()
    lines = {}
    launches = 0
    clocks = Clocks(dev.index)
    clocks.start()
    for which in sorted(S.PITCHED_LARGE):
        w = S.pitched_large(which)
        q = w.copies[0]
        n = q["width"] * q["height"] * q["depth"]
        a_dev = torch.from_numpy(w.image.a_bits[: w.image.n // 8].copy()).to(dev)
        v_dev = torch.from_numpy(w.image.v).to(dev)
        ctx = cg.Context()
        ctx.bind_host_shadow(a_dev, v_dev)
        for b, s_ in sorted(zip(w.table.base.tolist(), w.table.size.tolist())):
            cg.check(ctx.register_alloc(int(b), int(s_)), "register")
        qq = cg.copy3d(q["kind"], q["dst"], q["src"], q["width"], q["height"], q["depth"])
        rep = torch.zeros(cg.REPORT_DTYPE.itemsize, dtype=torch.uint8, device=dev)
        for _ in range(max(3, args.warmup)):
            cg.check(cg.cg_check_copy3d_async(ctx.handle, ctypes.byref(qq), rep.data_ptr(), sh),
                     "check3d")
        torch.cuda.synchronize()
        r = np.frombuffer(rep.cpu().numpy().tobytes(), dtype=cg.REPORT_DTYPE)[0]
        payload = np.lib.stride_tricks.as_strided(w.image.v, shape=(q["height"], q["width"]),
                                                  strides=(q["src"]["pitch"], 1))
        assert int(r["n_undef"]) == int((payload != 0).sum()), "report mismatch"
        # the checks run back to back as a user issues them; the region's
        # events give the mean launch duration (inter-launch gaps included),
        # and a second pass with events around every launch shows what
        # those extra event records cost
        k0 = ctx.stats()["kernels"]
        r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        r0.record(stream)
        for _ in range(args.steps):
            cg.check(cg.cg_check_copy3d_async(ctx.handle, ctypes.byref(qq), rep.data_ptr(), sh),
                     "check3d")
        r1.record(stream)
        torch.cuda.synchronize()
        launches += ctx.stats()["kernels"] - k0
        ms = r0.elapsed_time(r1) / args.steps
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        for e0, e1 in ev:
            e0.record(stream)
            cg.check(cg.cg_check_copy3d_async(ctx.handle, ctypes.byref(qq), rep.data_ptr(), sh),
                     "check3d")
            e1.record(stream)
        torch.cuda.synchronize()
        ms_each = float(np.mean([e0.elapsed_time(e1) for e0, e1 in ev]))
        achieved = BYTES_PER_BYTE_CARRY * n / (ms / 1e3) / GB
        span = (q["height"] - 1) * q["src"]["pitch"] + q["width"]
        lines[which] = {
            "checked_gb_per_s": round(n / (ms / 1e3) / GB, 2), "kernel_ms_mean": round(ms, 4),
            "kernel_ms_mean_events_per_launch": round(ms_each, 4),
            "payload_bytes": n, "host_span_bytes": span,
            "rows": q["height"], "row_bytes": q["width"], "host_pitch": q["src"]["pitch"],
            "dev_pitch": q["dst"]["pitch"], "n_undef_payload": int(r["n_undef"]),
            "roofline": {"bound": "hbm", "kernel": "scan_pitched_kernel<HTOD,carry>",
                         "bytes_per_checked_byte": BYTES_PER_BYTE_CARRY,
                         "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(achieved / peak, 4), "peak_source": peak_kind}}
        ctx.close()
        del a_dev, v_dev
        torch.cuda.empty_cache()
    clk = clocks.stop()
    out = {"metric": "pitched host->device checks: payload GB/s checked vs HBM peak",
           "unit": "GB/s", "value": min(d["checked_gb_per_s"] for d in lines.values()),
           "steps": args.steps, "warmup": max(3, args.warmup), "gpu_launches": int(launches),
           "config": {"workload": "pitched_large (wide 16 KiB rows, narrow 16 B of 24 B records)",
                      "l2": "inputs larger than L2 (>= 256 MiB each); no flush"},
           "lines": lines}
    if clk is not None:
        out["clocks"] = clk
    return out


def run_devops(args):
    """Memset and kernel-argument checks, timed with CUDA events: a 1 GiB
    memset (its shadow fill is 1 B written per byte), one launch with four
    256 MiB arguments (read scans 1 B read per byte, write fills 1 B written
    per byte), and the per-launch latency of checking the arguments of many
    small launches (1-6 arguments of 16 B - 64 KiB) against a table of
    100,000 allocations."""
    import torch

    import paper_1310_0901_gb300 as cg

    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream(dev)
    peak, peak_kind = _peaks()
    wl = S.devops_large()
    ctx = cg.Context()
    a_dev = torch.from_numpy(wl.image.a_bits[: wl.image.n // 8].copy()).to(dev)
    v_dev = torch.from_numpy(wl.image.v).to(dev)
    ctx.bind_host_shadow(a_dev, v_dev)
    for b, s_ in sorted(zip(wl.table.base.tolist(), wl.table.size.tolist())):
        cg.check(ctx.register_alloc(int(b), int(s_)), "register")
    for q in wl.setup:
        cg.check(ctx.check_copy(*q)[0], "setup")
    k0 = ctx.stats()["kernels"]
    clocks = Clocks(dev.index)
    clocks.start()

    def timed(fn, steps):
        for _ in range(max(3, args.warmup)):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    d, pitch, wd, h = wl.memset
    ms_memset = timed(lambda: cg.check(ctx.check_memset(d, wd, h, pitch, stream)[0], "memset"),
                      args.steps)
    n_set = wd * h
    ms_launch = timed(lambda: cg.check(ctx.check_kernel_args(wl.args, stream)[0], "args"),
                      args.steps)
    st, reps, _ = ctx.check_kernel_args(wl.args, stream)
    launches = ctx.stats()["kernels"] - k0
    moved = int(sum(int(x["bytes"]) for x in wl.args if x["access"] & S.ARG_READ)) + \
        int(sum(int(x["bytes"]) for x in wl.args if x["access"] & S.ARG_WRITE))
    ctx.close()
    del a_dev, v_dev
    torch.cuda.empty_cache()
    # many small launches over a 100k-entry table: host-timed latency per call
    rng = S.rng_for(77)
    table = S.alloc_table(rng, 100_000, 256, 1 << 20, True)
    small = S.kernel_launches(rng, 2000, table)
    ctx = cg.Context()
    order = np.argsort(table.base)
    st_ = ctx.register_allocs(table.base[order], table.size[order])
    assert not st_.any()
    for x in small[:50]:
        cg.check(ctx.check_kernel_args(x, stream)[0], "args")
    torch.cuda.synchronize()
    lat = []
    for x in small:
        t0 = time.perf_counter()
        cg.check(ctx.check_kernel_args(x, stream)[0], "args")
        lat.append((time.perf_counter() - t0) * 1e6)
    lat = np.array(lat)
    launches += ctx.stats()["kernels"]
    ctx.close()
    clk = clocks.stop()
    fill_gbs = n_set / (ms_memset / 1e3) / GB
    launch_gbs = moved / (ms_launch / 1e3) / GB
    out = {
        "metric": "memset / kernel-argument checks: shadow GB/s vs HBM peak; per-launch latency",
        "unit": "GB/s", "value": round(fill_gbs, 1), "steps": args.steps,
        "warmup": max(3, args.warmup), "gpu_launches": int(launches),
        "config": {"workload": "devops_large (1 GiB memset; 4 x 256 MiB arguments) + 2000 small "
                               "launches over 100k allocations",
                   "l2": "inputs larger than L2; no flush"},
        "memset": {"bytes": n_set, "ms": round(ms_memset, 4), "gb_per_s": round(fill_gbs, 1),
                   "roofline": {"bound": "hbm", "kernel": "fill_rows_kernel",
                                "bytes_per_byte": 1.0, "achieved": round(fill_gbs, 1),
                                "peak": peak, "unit": "GB/s",
                                "frac": round(fill_gbs / peak, 4), "peak_source": peak_kind}},
        "large_launch": {"args": len(wl.args), "bytes_read_plus_written": moved,
                         "ms": round(ms_launch, 4), "gb_per_s": round(launch_gbs, 1),
                         "roofline": {"bound": "hbm", "bytes_per_byte": 1.0,
                                      "achieved": round(launch_gbs, 1), "peak": peak,
                                      "unit": "GB/s", "frac": round(launch_gbs / peak, 4),
                                      "peak_source": peak_kind},
                         "n_undef": [int(r["n_undef"]) for r in reps]},
        "small_launches": {"launches": len(small), "table": 100_000,
                           "args_per_launch_mean": round(float(np.mean([len(x) for x in small])), 2),
                           "latency_us": {"p50": round(float(np.percentile(lat, 50)), 1),
                                          "p99": round(float(np.percentile(lat, 99)), 1)},
                           "launches_per_s": round(len(small) / (lat.sum() / 1e6), 1)},
    }
    if clk is not None:
        out["clocks"] = clk
    return out


def _baselines(d: dict) -> dict:
    return {k: d[k] for k in ("cpu_baseline", "cpu_baseline_all_cores") if k in d}


def _summary(key: str, d: dict) -> dict:
    if key == "devops":
        return {"workload": d["config"]["workload"],
                "memset_gb_per_s": d["memset"]["gb_per_s"],
                "memset_roofline_frac": d["memset"]["roofline"]["frac"],
                "large_launch_gb_per_s": d["large_launch"]["gb_per_s"],
                "large_launch_roofline_frac": d["large_launch"]["roofline"]["frac"],
                "small_launch_latency_us": d["small_launches"]["latency_us"]}
    if key == "pitched":
        return {"workload": d["config"]["workload"],
                **{k: {"checked_gb_per_s": v["checked_gb_per_s"],
                       "roofline_frac": v["roofline"]["frac"],
                       "kernel_ms_mean": v["kernel_ms_mean"]} for k, v in d["lines"].items()}}
    if key == "small":
        return {"workload": d["config"]["workload"], "checks_per_s": d["value"],
                "mode": d["mode"],
                "one_batch_at_a_time_checks_per_s": d["one_batch_at_a_time"]["checks_per_s"],
                "one_launch_per_copy_checks_per_s": d["one_launch_per_copy"]["checks_per_s"],
                "speedup_vs_one_launch_per_copy": d["speedup_vs_one_launch_per_copy"],
                **_baselines(d)}
    if key in ("batched", "adversarial"):
        out = {"workload": d["config"]["workload"], "checks_per_s": d["value"],
               "mode": d["mode"],
               "one_batch_at_a_time_checks_per_s": d["one_batch_at_a_time"]["checks_per_s"],
               "gb_per_s": d["batched_gb_per_s"],
               "one_launch_per_copy_checks_per_s": d["one_launch_per_copy"]["checks_per_s"],
               "speedup_vs_one_launch_per_copy": d["speedup_vs_one_launch_per_copy"],
               "levels_per_batch": d["config"]["levels_per_batch"],
               "roofline_frac": d["roofline"]["frac"],
               "roofline_frac_during_level_kernels": d["roofline"]["frac_during_level_kernels"],
               "ms_per_batch": d["ms_per_step"], "breakdown_ms": d["batch_breakdown_ms"],
               "split": d["split"]}
        if key == "adversarial":
            out["records_per_s"] = d["records_per_s"]
            out["records_per_batch"] = d["records_per_batch"]
        out.update(_baselines(d))
        return out
    return {"workload": d["config"]["workload"], "checks_per_s": d["value"],
            "latency_us": d["latency_us"], "offered_rate_per_s": d["config"]["offered_rate_per_s"],
            "all_ok": d["all_ok"], "rounds": d["serve_stats"]["rounds"],
            "rate_sweep": d["rate_sweep"], "one_launch_per_copy": d["one_launch_per_copy"],
            **({"speedup_vs_one_launch_per_copy": d["speedup_vs_one_launch_per_copy"]}
               if "speedup_vs_one_launch_per_copy" in d else {}),
            **_baselines(d)}


def _kernel_hash() -> str:
    """Hash of the headline kernel's sources with comments and blank lines
    dropped (a comment edit does not invalidate the captured traffic)."""
    import hashlib
    import re
    h = hashlib.sha1()
    for f in ("cg_scan_tma.cu", "cg_tma.cuh", "cg_device.cuh", "cg_internal.h"):
        text = open(os.path.join(ROOT, "paper_1310_0901_gb300", "csrc", f)).read()
        code = [ln.rstrip() for ln in (re.sub(r"//.*", "", x) for x in text.splitlines())]
        h.update("\n".join(ln for ln in code if ln.strip()).encode())
    return h.hexdigest()[:12]


def _profiled_traffic():
    """DRAM bytes per 4 GiB launch from the committed ncu summary, or None
    when the kernel sources changed since that capture."""
    import re
    p = os.path.join(ROOT, "profiles", "scan_single_tma_htod_1GiB_4GiB.md")
    if not os.path.exists(p):
        return None
    m = re.search(r"traffic_per_launch_bytes=(\d+); kernel_hash=(\w+)", open(p).read())
    if not m or m.group(2) != _kernel_hash():
        return None
    return int(m.group(1))


def cpu_sample(w, budget_s: float):
    """The oracle, as it stands, on a bounded sample of the same workload:
    host->device checks of the workload's transfers in order (smallest
    first) until the time budget is used; one thread."""
    import oracle as O
    sizes = sorted(int(q["n"]) for q in w.reqs)
    reqs = sorted(w.reqs, key=lambda q: int(q["n"]))
    n_img = sizes[-1]
    done = 0
    t = 0.0
    used = []
    img_n = min(n_img, max(sizes[0], 1 << 28))
    orc = O.Oracle(w.image.a_bits[: (img_n + 7) // 8], w.image.v[:img_n])
    order = np.argsort(w.table.base)
    for b, s in zip(w.table.base[order], w.table.size[order]):
        orc.register_alloc(int(b), int(s))
    while t < budget_s:
        q = reqs[0]
        n = min(int(q["n"]), img_n)
        s0 = time.perf_counter()
        st, _ = orc.check_copy(int(q["kind"]), int(q["dst"]), int(q["src"]), n)
        t += time.perf_counter() - s0
        assert st == 0
        done += n
        used.append(n)
    orc.close()
    return done / t / GB, f"{len(used)} x host->device check of {used[0] >> 20} MiB (first transfer of the workload), 1 thread, {t:.1f} s"


def cpu_sample_all_cores(w, budget_s: float):
    """The same oracle on all host cores: the smallest transfer of the
    workload is split into one part per thread, and every thread runs the
    oracle's host->device check on its own part (its own oracle state, the
    same per-byte code) until the time budget is used.  The calls into the
    oracle's C library release the interpreter lock, so the threads run in
    parallel.  Returns (GB/s over all threads, threads, sample text)."""
    import threading

    import oracle as O
    q = min(w.reqs, key=lambda r: int(r["n"]))
    n = int(q["n"])
    threads = max(1, len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity")
                  else (os.cpu_count() or 1))
    part = (n // threads) & ~4095
    orcs = []
    for t in range(threads):
        lo = t * part
        o = O.Oracle(w.image.a_bits[lo // 8:(lo + part) // 8], w.image.v[lo:lo + part])
        assert o.register_alloc(1 << 40, part) == 0
        orcs.append(o)
    done = [0] * threads
    spent = [0.0] * threads
    start = threading.Barrier(threads + 1)

    def work(t):
        o = orcs[t]
        start.wait()
        s0 = time.perf_counter()
        while time.perf_counter() - s0 < budget_s:
            st, _ = o.check_copy(S.HTOD, 1 << 40, 0, part)
            assert st == 0
            done[t] += part
        spent[t] = time.perf_counter() - s0

    pool = [threading.Thread(target=work, args=(t,)) for t in range(threads)]
    for th in pool:
        th.start()
    start.wait()
    for th in pool:
        th.join()
    for o in orcs:
        o.close()
    val = sum(done) / max(spent) / GB
    return val, threads, (f"{n >> 20} MiB host->device check split into {threads} parts of "
                          f"{part >> 20} MiB, one thread and one oracle state per part, "
                          f"{max(spent):.1f} s")


def _host_cores() -> int:
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)


def _cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.machine()


def _oracle_state(image, table, carry=True):
    """One oracle state over a workload's image and allocation table (its own
    copies of both; freed allocations freed)."""
    import oracle as O
    orc = O.Oracle(image.a_bits, image.v, carry=carry)
    order = np.argsort(table.base, kind="stable")
    assert not orc.register_allocs(table.base[order], table.size[order]).any()
    for j in table.freed:
        orc.free(int(table.base[j]))
    return orc


def oracle_copy_baselines(image, table, reqs, budget_s: float, what: str) -> dict:
    """The oracle, as it stands, timed on a bounded sample of a copy
    workload.  One thread: a prefix of the workload's requests, applied in
    order by one oracle state (one or_check_batch call, sized to take about
    the budget).  All cores: one oracle state per thread (its own image and
    table copies); thread t applies requests t, t + T, t + 2T, ... in order
    (one call, about half the budget).  Checks/s and checked GB/s."""
    import threading
    out = {}
    cpu = _cpu_model()
    orc = _oracle_state(image, table)
    # calibrate: bytes/s over the first requests
    k = 1
    while True:
        run = orc.batch_runner(reqs[:k])
        s0 = time.perf_counter()
        run()
        dt = time.perf_counter() - s0
        if dt > 0.2 or k >= len(reqs):
            break
        k = min(len(reqs), k * 4)
    rate = int(reqs["n"][:k].sum()) / dt
    orc.close()
    cum = np.cumsum(reqs["n"].astype(np.float64))
    m = max(1, min(len(reqs), int(np.searchsorted(cum, rate * budget_s)) + 1))
    orc = _oracle_state(image, table)
    run = orc.batch_runner(reqs[:m])
    s0 = time.perf_counter()
    assert run() == 0
    t = time.perf_counter() - s0
    orc.close()
    out["cpu_baseline"] = {
        "value": round(m / t, 1), "unit": "checks/s",
        "gb_per_s": round(float(cum[m - 1]) / t / GB, 4), "cores": 1, "kind": "oracle",
        "cpu": cpu,
        "sample": f"the first {m} requests of the {what} workload in order, one batch call, "
                  f"1 thread, {t:.1f} s"}
    cores = _host_cores()
    parts = [reqs[j::cores] for j in range(cores)]
    runs = [None] * cores
    states = [None] * cores

    def make(j):
        states[j] = _oracle_state(image, table)
        pc = np.cumsum(parts[j]["n"].astype(np.float64))
        mj = max(1, min(len(parts[j]), int(np.searchsorted(pc, rate * budget_s / 2)) + 1))
        parts[j] = parts[j][:mj]
        runs[j] = states[j].batch_runner(parts[j])

    pool = [threading.Thread(target=make, args=(j,)) for j in range(cores)]
    for th in pool:
        th.start()
    for th in pool:
        th.join()
    start = threading.Barrier(cores + 1)

    def work(j):
        start.wait()
        assert runs[j]() == 0

    pool = [threading.Thread(target=work, args=(j,)) for j in range(cores)]
    for th in pool:
        th.start()
    start.wait()
    s0 = time.perf_counter()
    for th in pool:
        th.join()
    wall = time.perf_counter() - s0
    for o in states:
        o.close()
    nchk = sum(len(x) for x in parts)
    nbyt = sum(int(x["n"].sum()) for x in parts)
    out["cpu_baseline_all_cores"] = {
        "value": round(nchk / wall, 1), "unit": "checks/s", "gb_per_s": round(nbyt / wall / GB, 4),
        "cores": cores, "kind": "oracle", "cpu": cpu,
        "sample": f"{nchk} requests of the {what} workload dealt round-robin to {cores} threads, "
                  f"each thread its own oracle state and one batch call, {wall:.1f} s"}
    return out


def run_reference(args, world, rank):
    """The reference arm: the CPU oracle on the host cores, rank 0 only."""
    if rank != 0:
        return None
    sizes = tuple(int(x) << 20 for x in args.sizes_mib.split(","))
    w = build_workload(sizes)
    import oracle as O
    n0 = min(int(q["n"]) for q in w.reqs)
    orc = O.Oracle(w.image.a_bits[: n0 // 8], w.image.v[:n0])
    order = np.argsort(w.table.base)
    for b, s in zip(w.table.base[order], w.table.size[order]):
        orc.register_alloc(int(b), int(s))
    q = min(w.reqs, key=lambda r: int(r["n"]))
    sample = min(int(q["n"]), 64 << 20)  # each step: the first 64 MiB of the smallest transfer
    for _ in range(args.warmup):
        orc.check_copy(int(q["kind"]), int(q["dst"]), int(q["src"]), sample)
    s0 = time.perf_counter()
    for _ in range(args.steps):
        st, _ = orc.check_copy(int(q["kind"]), int(q["dst"]), int(q["src"]), sample)
        assert st == 0
    dt = time.perf_counter() - s0
    val = sample * args.steps / dt / GB
    orc.close()
    return {
        "impl": "reference",
        "metric": "shadow GB/s checked vs HBM peak (single large host->device transfer checks)",
        "value": round(val, 4), "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic", "config": {"workload": w.name, "parallelism": "cpu oracle, 1 thread"},
        "cpu_baseline": {"value": round(val, 4), "unit": "GB/s", "cores": 1, "kind": "oracle",
                         "sample": f"first {sample >> 20} MiB of the {int(q['n']) >> 20} MiB "
                                   "host->device check per step"},
        "e2e": {"value": round(val, 4), "unit": "GB/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="cg", choices=["cg", "reference"])
    ap.add_argument("--sizes-mib", default="256,1024,4096")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--cpu-budget-s", type=float, default=10.0)
    ap.add_argument("--engine", type=int, default=0, help="0 auto, 1 register loads, 2 TMA bulk")
    ap.add_argument("--workload", default="large",
                    choices=["large", "small", "batched", "adversarial", "serving", "pitched",
                             "devops"])
    ap.add_argument("--serve-seconds", type=float, default=10.0)
    ap.add_argument("--serve-rate", type=float, default=S.SERVE_RATE)
    ap.add_argument("--serve-image-gib", type=int, default=32)
    ap.add_argument("--serve-streams", type=int, default=4)
    ap.add_argument("--extras", type=int, default=1,
                    help="1: add the batched and serving figures to the default line")
    ap.add_argument("--segment-kib", type=int, default=0)
    ap.add_argument("--piece-kib", type=int, default=0,
                    help="batch_piece_kib: 0 = the library's default, 4294967295 = whole copies")
    ap.add_argument("--single-sample", type=int, default=100_000)
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    world, rank, local = _dist()
    if args.impl == "reference":
        out = run_reference(args, world, rank)
        if out is not None:
            print(json.dumps(out), flush=True)
        return
    if args.workload == "serving":
        if rank == 0:
            print(json.dumps(run_serving(args)), flush=True)
        return
    if args.workload in ("pitched", "devops", "small"):
        if rank == 0:
            fn = {"pitched": run_pitched, "devops": run_devops, "small": run_small}[args.workload]
            print(json.dumps(fn(args)), flush=True)
        return
    if args.workload != "large":
        if rank == 0:
            print(json.dumps(run_batched_workload(args, args.workload)), flush=True)
        return
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    out, w = run_cg(args, world, rank, local)
    if rank == 0:
        if world == 1 and args.cpu_budget_s > 0:
            val, sample = cpu_sample(w, args.cpu_budget_s)
            out["cpu_baseline"] = {"value": round(val, 4), "unit": "GB/s", "cores": 1,
                                   "kind": "oracle", "sample": sample}
            val, threads, sample = cpu_sample_all_cores(w, args.cpu_budget_s / 2)
            out["cpu_baseline_all_cores"] = {"value": round(val, 4), "unit": "GB/s",
                                             "cores": threads, "kind": "oracle",
                                             "sample": sample}
        if world == 1 and args.extras:
            # the metric's other two parts, on their own workloads (batched
            # checks/s against one launch per copy; serving latency)
            import torch
            del w
            torch.cuda.empty_cache()
            for key, fn in (("small", lambda: run_small(args)),
                            ("batched", lambda: run_batched_workload(args, "batched")),
                            ("adversarial", lambda: run_batched_workload(args, "adversarial")),
                            ("serving", lambda: run_serving(args)),
                            ("pitched", lambda: run_pitched(args)),
                            ("devops", lambda: run_devops(args))):
                t_key = time.perf_counter()
                try:
                    out[key] = _summary(key, fn())
                except Exception as exc:  # reported, never hides the headline
                    out[key] = {"error": f"{type(exc).__name__}: {exc}"}
                print(f"[bench] {key}: {time.perf_counter() - t_key:.1f} s", file=sys.stderr,
                      flush=True)
                torch.cuda.empty_cache()
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()

"""Seeded synthetic inputs for the transfer checks.

This module only *produces inputs*: host shadow images (packed addressability
bitmap + per-byte definedness masks), device allocation tables and copy
request streams, each with the ground truth of what was planted.  It holds
none of the checking arithmetic, and both the GPU library's tests and the CPU
oracle draw their inputs from here.

Layouts (the same ones the library documents):
  * A bitmap: 1 bit per host byte, byte ``p`` <-> bit ``p & 7`` of
    ``a_bits[p >> 3]``, 1 = addressable (``np.packbits(..., 'little')``).
  * V mask: 1 byte per host byte, bit set = that data bit is undefined.
  * requests: ``REQ_DTYPE`` records (kind, reserved, dst, src, n); for a
    host->device copy ``src`` is an offset into the host image, for a
    device->host copy ``dst`` is.

All draws use numpy's PCG64 generator, which gives identical streams on x86
and Arm hosts.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

HTOD, DTOH, DTOD = 1, 2, 3
REQ_DTYPE = np.dtype([("kind", "<u4"), ("reserved", "<u4"), ("dst", "<u8"),
                      ("src", "<u8"), ("n", "<u8")])
ADDR_SPACE = 1 << 48


@dataclass
class HostImage:
    a_bits: np.ndarray            # uint8, ceil(n/8) bytes (padded to 16)
    v: np.ndarray                 # uint8, n bytes
    undef_runs: list = field(default_factory=list)   # (start, length) planted
    unaddr: np.ndarray | None = None                 # planted positions (sorted)

    @property
    def n(self) -> int:
        return int(self.v.size)


@dataclass
class AllocTable:
    base: np.ndarray              # uint64
    size: np.ndarray              # uint64
    freed: np.ndarray             # indices into base/size freed after registration


def rng_for(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def pack_a(addressable: np.ndarray) -> np.ndarray:
    """bool per byte -> packed LSB-first bitmap, padded to a 16-byte multiple."""
    bits = np.packbits(addressable.astype(np.uint8), bitorder="little")
    pad = (-bits.size) % 16
    if pad:
        bits = np.concatenate([bits, np.zeros(pad, np.uint8)])
    return bits


def log_uniform_int(rng, lo: int, hi: int, size) -> np.ndarray:
    """Integers log-uniform on [lo, hi]."""
    x = np.exp(rng.uniform(np.log(lo), np.log(hi + 1), size=size))
    return np.clip(np.floor(x), lo, hi).astype(np.uint64)


def partial_masks(rng, count: int) -> np.ndarray:
    """Random nonzero definedness masks other than 0xFF."""
    return rng.integers(1, 255, size=count, dtype=np.uint8)


def host_image_runs(rng, n: int, undef_frac: float, mean_run: float = 8.0,
                    partial_frac: float = 0.5, unaddr_p: float = 0.0) -> HostImage:
    """Undefined bytes planted as runs of geometric length until ``undef_frac``
    of the bytes are covered; each run is fully undefined (0xFF) or carries
    random partial masks.  Unaddressable bytes are Bernoulli(unaddr_p)."""
    v = np.zeros(n, dtype=np.uint8)
    runs = []
    target = int(round(undef_frac * n))
    covered = 0
    while covered < target and n > 0:
        length = int(min(rng.geometric(1.0 / mean_run), n))
        start = int(rng.integers(0, n - length + 1))
        if rng.random() < partial_frac:
            v[start:start + length] = partial_masks(rng, length)
        else:
            v[start:start + length] = 0xFF
        runs.append((start, length))
        covered += length
    if unaddr_p > 0:
        k = rng.binomial(n, unaddr_p)
        unaddr = np.unique(rng.integers(0, n, size=k))
    else:
        unaddr = np.zeros(0, dtype=np.int64)
    addressable = np.ones(n, dtype=bool)
    addressable[unaddr] = False
    return HostImage(pack_a(addressable), v, runs, unaddr)


def host_image_dense(rng, n: int, partial_p: float, unaddr_p: float,
                     chunk: int = 1 << 26) -> HostImage:
    """Every byte independently carries a random partial mask with
    probability ``partial_p`` and is unaddressable with probability
    ``unaddr_p`` (the adversarial-density workload)."""
    v = np.empty(n, dtype=np.uint8)
    a_bits = np.empty((n + 7) // 8, dtype=np.uint8)
    for lo in range(0, n, chunk):
        hi = min(n, lo + chunk)
        m = hi - lo
        has = rng.random(m) < partial_p
        v[lo:hi] = np.where(has, rng.integers(1, 255, size=m, dtype=np.uint8), 0)
        addr = rng.random(m) >= unaddr_p
        a_bits[lo // 8:(hi + 7) // 8] = np.packbits(addr.astype(np.uint8), bitorder="little")
    pad = (-a_bits.size) % 16
    if pad:
        a_bits = np.concatenate([a_bits, np.zeros(pad, np.uint8)])
    return HostImage(a_bits, v, [], None)


def host_image_clean(n: int) -> HostImage:
    return HostImage(pack_a(np.ones(n, dtype=bool)), np.zeros(n, dtype=np.uint8), [],
                     np.zeros(0, dtype=np.int64))


def disjoint_bases(rng, sizes: np.ndarray, align: int = 256,
                   space: int = ADDR_SPACE) -> np.ndarray:
    """Random, ``align``-aligned, pairwise disjoint bases in [0, space): the
    space is cut into one slot per allocation (slots shuffled) and each
    allocation lands at a random aligned offset inside its slot."""
    k = len(sizes)
    slot = space // k
    slot -= slot % align
    assert int(sizes.max()) <= slot, "allocations larger than their slots"
    order = rng.permutation(k).astype(np.uint64)
    room = (slot - sizes.astype(np.uint64)) // align
    off = (rng.random(k) * (room.astype(np.float64) + 1)).astype(np.uint64) * align
    return order * np.uint64(slot) + off


def alloc_table(rng, count: int, size_lo: int, size_hi: int, log_sizes: bool,
                n_freed: int = 0, round_to: int = 1) -> AllocTable:
    if log_sizes:
        sizes = log_uniform_int(rng, size_lo, size_hi, count)
    else:
        sizes = rng.integers(size_lo, size_hi + 1, size=count).astype(np.uint64)
    if round_to > 1:
        sizes = ((sizes + np.uint64(round_to - 1)) // np.uint64(round_to)) * np.uint64(round_to)
    bases = disjoint_bases(rng, sizes)
    freed = rng.choice(count, size=n_freed, replace=False) if n_freed else np.zeros(0, np.int64)
    return AllocTable(bases.astype(np.uint64), sizes.astype(np.uint64), np.sort(freed))


def _device_target(rng, table: AllocTable, live_idx: np.ndarray, n: int,
                   p_freed: float, p_overrun: float, p_wild: float) -> int:
    u = rng.random()
    if u < p_freed and table.freed.size:
        j = int(table.freed[rng.integers(0, table.freed.size)])
        return int(table.base[j]) + int(rng.integers(0, int(table.size[j])))
    u -= p_freed
    if u < p_wild:
        return int(rng.integers(0, ADDR_SPACE))
    u -= p_wild
    j = int(live_idx[rng.integers(0, live_idx.size)])
    base, size = int(table.base[j]), int(table.size[j])
    if u < p_overrun and n >= 2:
        k = int(rng.integers(1, min(n - 1, size) + 1))
        return base + size - k
    if n <= size:
        return base + int(rng.integers(0, size - n + 1))
    return base


def requests(rng, count: int, table: AllocTable, host_n: int, n_lo: int, n_hi: int,
             mix=(0.6, 0.3, 0.1), p_freed: float = 0.0, p_overrun: float = 0.0,
             p_wild: float = 0.0, p_same_alloc_dtod: float = 0.1) -> np.ndarray:
    """A copy stream: kinds drawn from ``mix`` (HtoD, DtoH, DtoD), sizes
    log-uniform in [n_lo, n_hi] (capped at the host image), host offsets
    uniform, device targets inside live allocations except for the planted
    overruns, freed-pointer targets and wild pointers."""
    live = np.setdiff1d(np.arange(len(table.base)), table.freed)
    reqs = np.zeros(count, dtype=REQ_DTYPE)
    kinds = rng.choice([HTOD, DTOH, DTOD], size=count, p=list(mix))
    sizes = log_uniform_int(rng, n_lo, n_hi, count)
    for i in range(count):
        kind = int(kinds[i])
        n = int(min(int(sizes[i]), host_n)) if kind != DTOD else int(sizes[i])
        reqs[i]["kind"] = kind
        reqs[i]["n"] = n
        if kind == HTOD:
            reqs[i]["src"] = int(rng.integers(0, host_n - n + 1))
            reqs[i]["dst"] = _device_target(rng, table, live, n, p_freed, p_overrun, p_wild)
        elif kind == DTOH:
            reqs[i]["dst"] = int(rng.integers(0, host_n - n + 1))
            reqs[i]["src"] = _device_target(rng, table, live, n, p_freed, p_overrun, p_wild)
        else:
            s = _device_target(rng, table, live, n, p_freed, p_overrun, p_wild)
            if rng.random() < p_same_alloc_dtod:
                # destination a few bytes away from the source: exercises
                # overlapping device->device copies
                k = min(n, 64)
                d = max(s + int(rng.integers(-k, k + 1)), 0)
            else:
                d = _device_target(rng, table, live, n, p_freed, p_overrun, p_wild)
            reqs[i]["src"] = s
            reqs[i]["dst"] = d
    return reqs


# ----------------------------------------------------------------- configs

@dataclass
class Workload:
    name: str
    image: HostImage
    table: AllocTable
    reqs: np.ndarray
    note: str = ""


def small(seed: int = 0) -> Workload:
    """64 live device allocations (72 registered, 8 freed), sizes uniform
    1-16 KiB rounded to 256 B; 1 MiB host image, 1 % undefined bytes in runs
    of geometric mean length 8 (half partial masks), 0.1 % unaddressable;
    1,000 requests 60/30/10 HtoD/DtoH/DtoD, sizes log-uniform 1 B-16 KiB,
    10 % overrunning, 2 % aimed at freed allocations."""
    rng = rng_for(seed)
    table = alloc_table(rng, 72, 1, 16 * 1024, log_sizes=False, n_freed=8, round_to=256)
    img = host_image_runs(rng, 1 << 20, 0.01, 8.0, 0.5, 0.001)
    reqs = requests(rng, 1000, table, img.n, 1, 16 * 1024, p_freed=0.02, p_overrun=0.10,
                    p_wild=0.01)
    return Workload("small-1k-requests-1MiB-image", img, table, reqs)


LARGE_SIZES = (256 << 20, 1 << 30, 4 << 30)


def large(seed: int = 0, sizes=LARGE_SIZES) -> Workload:
    """Large single host->device transfers (default 256 MiB, 1 GiB, 4 GiB)
    from one host image of the largest size, undefined density 1e-6 in sparse
    runs, fully addressable, against a 16-entry allocation table in which one
    allocation per transfer holds the destination at offset 0."""
    rng = rng_for(seed)
    n_img = int(max(sizes))
    img = host_image_runs(rng, n_img, 1e-6, 8.0, 0.5, 0.0)
    small_sizes = rng.integers(4096, 1 << 20, size=16 - len(sizes)).astype(np.uint64)
    all_sizes = np.concatenate([np.array(sizes, dtype=np.uint64), small_sizes])
    bases = disjoint_bases(rng, all_sizes, align=1 << 16)
    table = AllocTable(bases, all_sizes, np.zeros(0, np.int64))
    reqs = np.zeros(len(sizes), dtype=REQ_DTYPE)
    for i, n in enumerate(sizes):
        reqs[i] = (HTOD, 0, int(bases[i]), 0, int(n))
    return Workload("large-htod-" + "-".join(_human(s) for s in sizes), img, table, reqs)


def batched(seed: int = 0, n_req: int = 100_000, n_alloc: int = 1_000_000,
            host_n: int = 1 << 30, n_hi: int = 64 << 20) -> Workload:
    """100,000 requests, sizes log-uniform 16 B-64 MiB, against 1,000,000
    allocations log-uniform 256 B-1 MiB; 1 GiB host image, 0.01 % undefined."""
    rng = rng_for(seed)
    table = alloc_table(rng, n_alloc, 256, 1 << 20, log_sizes=True)
    img = host_image_runs(rng, host_n, 1e-4, 8.0, 0.5, 1e-5)
    reqs = requests(rng, n_req, table, host_n, 16, n_hi, p_wild=0.01)
    return Workload(f"batched-{n_req}-req-{n_alloc}-allocs", img, table, reqs)


def adversarial(seed: int = 0, n_req: int = 10_000, host_n: int = 1 << 30,
                n_alloc: int = 1024) -> Workload:
    """10,000 copies of 4 KiB-16 MiB over a host image where 50 % of the
    bytes carry random partial masks and 5 % are unaddressable; 1,024
    allocations log-uniform 4 KiB-32 MiB."""
    rng = rng_for(seed)
    table = alloc_table(rng, n_alloc, 4096, 32 << 20, log_sizes=True)
    img = host_image_dense(rng, host_n, 0.5, 0.05)
    reqs = requests(rng, n_req, table, host_n, 4096, 16 << 20)
    return Workload(f"adversarial-{n_req}-req", img, table, reqs)


def _human(n: int) -> str:
    for unit, sh in (("GiB", 30), ("MiB", 20), ("KiB", 10)):
        if n >= 1 << sh and n % (1 << sh) == 0:
            return f"{n >> sh}{unit}"
    return f"{n}B"


# ----------------------------------------------------------------- serving

OP_CHECK, OP_ALLOC, OP_FREE, OP_MARK_DEFINED, OP_MARK_UNDEFINED = 1, 2, 3, 4, 5
SERVE_DTYPE = np.dtype([("op", "<u4"), ("kind", "<u4"), ("dst", "<u8"), ("src", "<u8"),
                        ("n", "<u8")])


@dataclass
class ServeTrace:
    reqs: np.ndarray        # SERVE_DTYPE
    client: np.ndarray      # uint32
    arrival_ns: np.ndarray  # uint64, nondecreasing
    table: AllocTable       # allocations live before the trace starts
    note: str = ""


def serve_trace(rng, n_req: int, rate: float, clients: int, table: AllocTable, host_n: int,
                big: np.ndarray | None = None, event_frac: float = 0.05,
                size_mix=((0.80, 1, 4096), (0.19, 4096, 1 << 20), (0.01, 1 << 20, 256 << 20)),
                dyn_slots_per_client: int = 512, dyn_size=(256, 64 << 10),
                mark_frac: float = 0.0) -> ServeTrace:
    """Poisson arrivals at `rate` requests/s spread over `clients` streams.
    A fraction `event_frac` are allocation events (half allocations, half
    frees) on each client's own pool of address slots, so every client's
    frees follow its own allocations; the rest are checks (60/30/10
    HtoD/DtoH/DtoD) of the size classes in `size_mix` against the
    allocations of `table` (the largest class against `big`, the indices of
    large allocations, when given).  A fraction `mark_frac` of the checks
    becomes mark-defined/undefined requests."""
    gaps = rng.exponential(1.0 / rate, n_req)
    arrival = np.cumsum(gaps) * 1e9
    client = rng.integers(0, clients, n_req).astype(np.uint32)
    reqs = np.zeros(n_req, SERVE_DTYPE)
    is_event = rng.random(n_req) < event_frac
    # checks, vectorised
    kinds = rng.choice([HTOD, DTOH, DTOD], size=n_req, p=[0.6, 0.3, 0.1]).astype(np.uint32)
    cls = rng.choice(len(size_mix), size=n_req, p=[c[0] for c in size_mix])
    sizes = np.zeros(n_req, np.uint64)
    for k, (_, lo, hi) in enumerate(size_mix):
        m = cls == k
        sizes[m] = log_uniform_int(rng, lo, hi, int(m.sum()))
    sizes = np.minimum(sizes, np.uint64(host_n))
    live = np.arange(len(table.base))
    tgt = live[rng.integers(0, live.size, n_req)]
    if big is not None and big.size:
        bigm = cls == len(size_mix) - 1
        tgt[bigm] = big[rng.integers(0, big.size, int(bigm.sum()))]
    tsize = table.size[tgt].astype(np.uint64)
    room = np.where(sizes <= tsize, tsize - sizes, 0).astype(np.float64)
    off = (rng.random(n_req) * (room + 1)).astype(np.uint64)
    dev = table.base[tgt].astype(np.uint64) + off
    tgt2 = live[rng.integers(0, live.size, n_req)]
    tsize2 = table.size[tgt2].astype(np.uint64)
    room2 = np.where(sizes <= tsize2, tsize2 - sizes, 0).astype(np.float64)
    dev2 = table.base[tgt2].astype(np.uint64) + (rng.random(n_req) * (room2 + 1)).astype(np.uint64)
    host = (rng.random(n_req) * (host_n - sizes.astype(np.float64) + 1)).astype(np.uint64)
    reqs["op"] = OP_CHECK
    reqs["kind"] = kinds
    reqs["n"] = sizes
    reqs["dst"] = np.where(kinds == DTOH, host, dev)
    reqs["src"] = np.where(kinds == HTOD, host, np.where(kinds == DTOD, dev2, dev))
    if mark_frac > 0:
        mk = (~is_event) & (rng.random(n_req) < mark_frac)
        reqs["op"][mk] = np.where(rng.random(int(mk.sum())) < 0.5, OP_MARK_DEFINED,
                                  OP_MARK_UNDEFINED)
        reqs["dst"][mk] = dev[mk]
        reqs["src"][mk] = 0
        reqs["n"][mk] = np.minimum(sizes[mk], tsize[mk] - np.minimum(off[mk], tsize[mk]))
    # allocation events: each client owns a pool of address slots above the table
    top = int(table.base.max() + table.size.max()) if len(table.base) else 0
    slot_span = 1 << 20
    region = ((top >> 30) + 1) << 30
    live_dyn = [[] for _ in range(clients)]
    free_dyn = [list(range(dyn_slots_per_client)) for _ in range(clients)]
    for i in np.nonzero(is_event)[0]:
        c = int(client[i])
        if live_dyn[c] and (rng.random() < 0.5 or not free_dyn[c]):
            k = live_dyn[c].pop(int(rng.integers(0, len(live_dyn[c]))))
            free_dyn[c].append(k)
            reqs[i] = (OP_FREE, 0, region + (c * dyn_slots_per_client + k) * slot_span, 0, 0)
        else:
            k = free_dyn[c].pop(int(rng.integers(0, len(free_dyn[c]))))
            live_dyn[c].append(k)
            size = int(log_uniform_int(rng, dyn_size[0], dyn_size[1], 1)[0])
            reqs[i] = (OP_ALLOC, 0, region + (c * dyn_slots_per_client + k) * slot_span, 0, size)
    return ServeTrace(reqs, client, arrival.astype(np.uint64), table)


SERVE_RATE = 200_000.0


def serving(seed: int = 0, seconds: float = 10.0, rate: float = SERVE_RATE, clients: int = 8,
            host_n: int = 32 << 30, n_alloc: int = 100_000, n_big: int = 100) -> ServeTrace:
    """Poisson arrivals from 8 client streams at 200k requests/s: 80 % of
    the checks 1 B-4 KiB, 19 % 4 KiB-1 MiB, 1 % 1 MiB-256 MiB; allocation
    events 5 % of the traffic; 100,000 live allocations (log-uniform
    256 B-1 MiB) plus 100 of 256 MiB for the largest copies; a 32 GiB host
    image (described, not materialised: see serving_image_runs)."""
    rng = rng_for(seed)
    small_sizes = log_uniform_int(rng, 256, 1 << 20, n_alloc)
    sizes = np.concatenate([small_sizes, np.full(n_big, 256 << 20, np.uint64)])
    bases = disjoint_bases(rng, sizes, space=1 << 47)
    table = AllocTable(bases.astype(np.uint64), sizes.astype(np.uint64), np.zeros(0, np.int64))
    n_req = int(seconds * rate)
    tr = serve_trace(rng, n_req, rate, clients, table, host_n,
                     big=np.arange(n_alloc, n_alloc + n_big))
    tr.note = f"serving-{clients}-clients-{int(rate)}-req-per-s-{seconds}s-{host_n >> 30}GiB-image"
    return tr


def serving_image_runs(seed: int, host_n: int, undef_frac: float = 1e-5, mean_run: float = 8.0):
    """Planted undefined runs of a large host image, without materialising
    it: (starts, lengths, values) with values a nonzero mask per run."""
    rng = rng_for(seed + 1)
    k = max(1, int(undef_frac * host_n / mean_run))
    starts = rng.integers(0, host_n - 64, k).astype(np.int64)
    lengths = np.minimum(rng.geometric(1.0 / mean_run, k), 64).astype(np.int64)
    values = rng.integers(1, 256, k).astype(np.uint8)
    return starts, lengths, values


def tuning_batch(rng, table: AllocTable, host_n: int) -> np.ndarray:
    """A batch of random shape for fitting the split cost model: count
    500-8000, sizes log-uniform in [lo, hi] with lo 16 B-64 KiB and hi up to
    16 MiB, a random kind mix."""
    count = int(np.exp(rng.uniform(np.log(500), np.log(8000))))
    lo = int(2 ** rng.uniform(4, 16))
    hi = int(min(16 << 20, lo * 2 ** rng.uniform(2, 14)))
    mix = rng.dirichlet([2.0, 1.0, 0.5])
    return requests(rng, count, table, host_n, lo, max(lo, hi), mix=tuple(mix), p_wild=0.01)


def tuning_batch_mixed(rng, table: AllocTable, host_n: int) -> np.ndarray:
    """A batch from one of four shape families, for fitting and testing the
    split cost model on shapes where split sizes differ: tuning_batch's
    random shapes; a few large copies (16-200 of 1-16 MiB); a bimodal mix
    (500-4000 copies up to 4 KiB plus 10-200 of 1-16 MiB); mid-sized copies
    (200-2000 of 64 KiB-1 MiB)."""
    fam = int(rng.integers(0, 4))
    if fam == 0:
        return tuning_batch(rng, table, host_n)
    if fam == 1:
        return requests(rng, int(rng.integers(16, 200)), table, host_n, 1 << 20, 16 << 20)
    if fam == 2:
        a = requests(rng, int(rng.integers(500, 4000)), table, host_n, 16, 4096)
        b = requests(rng, int(rng.integers(10, 200)), table, host_n, 1 << 20, 16 << 20)
        q = np.concatenate([a, b])
        return q[rng.permutation(len(q))]
    return requests(rng, int(rng.integers(200, 2000)), table, host_n, 64 << 10, 1 << 20)


# ------------------------------------------------ pitched copies, arrays

@dataclass
class PitchedWorkload:
    image: HostImage
    table: AllocTable
    arrays: list  # (handle, width_bytes, height, depth)
    copies: list  # dicts: kind, dst, src (side dicts), width, height, depth
    name: str = ""


def side3d(ptr: int, pitch: int = 0, rows: int = 0, x: int = 0, y: int = 0, z: int = 0,
           array: bool = False) -> dict:
    return dict(ptr=int(ptr), pitch=int(pitch), rows=int(rows), x=int(x), y=int(y), z=int(z),
                is_array=int(array))


def _pitched_shape(rng, max_bytes: int):
    """Row width, rows and slices: narrow (record-like), medium and wide rows."""
    u = rng.random()
    if u < 0.35:
        w = int(rng.integers(1, 65))
    elif u < 0.7:
        w = int(rng.integers(65, 2049))
    else:
        w = int(rng.integers(2049, 24 * 1024))
    h = int(rng.integers(1, 65))
    d = int(rng.integers(1, 5)) if rng.random() < 0.3 else 1
    while w * h * d > max_bytes and h > 1:
        h = max(1, h // 2)
    if w * h * d > max_bytes:
        d = 1
    return w, h, d


def _pitch_for(rng, w: int) -> int:
    """A pitch >= w: tight, a small ragged gap, or rounded up to 512 B (the
    kind a pitched allocator returns)."""
    u = rng.random()
    if u < 0.2:
        return w
    if u < 0.6:
        return w + int(rng.integers(1, 80))
    return ((w + 511) // 512) * 512 + (512 if rng.random() < 0.3 else 0)


def _linear_side(rng, w, h, d, lo: int, room: int, p_over: float = 0.0):
    """A linear side whose extent starts in [lo, lo+room) and fits, or (with
    probability p_over) runs past lo+room."""
    pitch = _pitch_for(rng, w)
    rows = h + (int(rng.integers(0, 4)) if d > 1 else 0)
    x, y, z = int(rng.integers(0, 33)), int(rng.integers(0, 3)), int(rng.integers(0, 2))
    place = (z * rows + y) * pitch + x
    ext = ((d - 1) * rows + (h - 1)) * pitch + w
    if ext + place > room:
        x = y = z = 0
        place = 0
    if ext > room:
        return None
    if rng.random() < p_over:
        first = room - ext + int(rng.integers(1, min(ext, 4096) + 1))
    else:
        first = int(rng.integers(0, room - ext + 1))
    ptr = lo + max(first - place, 0)
    if first < place:  # keep the origin arithmetic inside [lo, ...)
        x = y = z = 0
        ptr = lo + first
    return side3d(ptr, pitch, rows, x, y, z)


def pitched(seed: int = 0, n_copies: int = 300, host_n: int = 8 << 20, max_bytes: int = 256 << 10,
            n_alloc: int = 48, n_arrays: int = 6) -> PitchedWorkload:
    """Pitched 2-D / 3-D copies over linear allocations (4 KiB - 4 MiB,
    log-uniform) and device arrays: kind mix 60/30/10, row widths from
    1 B (record fields) to 24 KiB, pitches tight, ragged or 512-rounded;
    10 % of linear device sides overrun, 3 % aim at a freed allocation,
    20 % of device sides are arrays (15 % of those boxes do not fit)."""
    rng = rng_for(7000 + seed)
    image = host_image_runs(rng, host_n, undef_frac=2e-3, mean_run=8.0, unaddr_p=5e-4)
    table = alloc_table(rng, n_alloc, 4096, 4 << 20, True, n_freed=3, round_to=256)
    live = np.setdiff1d(np.arange(n_alloc), table.freed)
    arrays = []
    for k in range(n_arrays):
        W = int(rng.integers(16, 4097))
        H = int(rng.integers(1, 129))
        D = int(rng.integers(1, 9)) if k % 2 else 1
        arrays.append((0x5000_0000 + 0x100 * k, W, H, D))
    copies = []
    while len(copies) < n_copies:
        kind = int(rng.choice([HTOD, DTOH, DTOD], p=[0.6, 0.3, 0.1]))
        w, h, d = _pitched_shape(rng, max_bytes)
        sides = {}
        ok = True
        for role in ("dst", "src"):
            host_side = (role == "src" and kind == HTOD) or (role == "dst" and kind == DTOH)
            if host_side:
                s = _linear_side(rng, w, h, d, 0, host_n)
            elif rng.random() < 0.2:
                handle, W, H, D = arrays[int(rng.integers(0, len(arrays)))]
                if rng.random() < 0.85 and w <= W and h <= H and d <= D:
                    x, y, z = (int(rng.integers(0, W - w + 1)), int(rng.integers(0, H - h + 1)),
                               int(rng.integers(0, D - d + 1)))
                else:
                    x, y, z = (int(rng.integers(0, W)), int(rng.integers(0, H)),
                               int(rng.integers(0, D)))
                s = side3d(handle, 0, 0, x, y, z, array=True)
            else:
                u = rng.random()
                j = int(rng.choice(table.freed)) if u < 0.03 and len(table.freed) else \
                    int(rng.choice(live))
                s = _linear_side(rng, w, h, d, int(table.base[j]), int(table.size[j]),
                                 p_over=0.1)
            if s is None:
                ok = False
                break
            sides[role] = s
        if not ok:
            continue
        if kind == DTOD and rng.random() < 0.3 and not sides["dst"]["is_array"]:
            # overlapping: the source shifted a little from the destination
            s = dict(sides["dst"])
            s["ptr"] = max(0, s["ptr"] + int(rng.integers(-300, 300)))
            sides["src"] = s
        copies.append(dict(kind=kind, dst=sides["dst"], src=sides["src"], width=w, height=h,
                           depth=d))
    return PitchedWorkload(image, table, arrays, copies, f"pitched/seed{seed}")


# Full-size pitched transfers (host->device with carry), 256 MiB of payload each:
#   wide:   16384 rows of 16 KiB, host and device pitch 16.5 KiB (512 B of
#           never-written padding per host row), as an image or matrix with a
#           padded leading dimension;
#   narrow: one 16-byte field of 16M 24-byte host records (8 B of never-written
#           padding each) into a dense device array: the strided host read of
#           the paper's footnote.
PITCHED_LARGE = {
    "wide": dict(width=16 << 10, height=16384, host_pitch=(16 << 10) + 512,
                 dev_pitch=(16 << 10) + 512),
    "narrow": dict(width=16, height=16 << 20, host_pitch=24, dev_pitch=16),
}


def pitched_large(which: str = "wide", seed: int = 0) -> PitchedWorkload:
    cfg = PITCHED_LARGE[which]
    w, h, hp, dp = cfg["width"], cfg["height"], cfg["host_pitch"], cfg["dev_pitch"]
    rng = rng_for(8000 + seed)
    host_ext = (h - 1) * hp + w
    host_n = (host_ext + 4095) // 4096 * 4096
    image = host_image_runs(rng, host_n, undef_frac=1e-6, mean_run=8.0)
    # the padding between rows was never written: undefined
    pad = np.ones(hp, bool)
    pad[:w] = False
    rows_in_image = host_n // hp
    view = image.v[: rows_in_image * hp].reshape(rows_in_image, hp)
    view[:, pad] = 0xFF
    image.v[rows_in_image * hp:] = 0xFF
    dev_size = (h - 1) * dp + w
    dev_size = (dev_size + 255) // 256 * 256
    sizes = np.array([dev_size] + [1 << 20] * 15, dtype=np.uint64)
    bases = disjoint_bases(rng, sizes)
    table = AllocTable(bases, sizes, np.zeros(0, np.int64))
    copy = dict(kind=HTOD, dst=side3d(int(bases[0]), dp, h), src=side3d(0, hp, h), width=w,
                height=h, depth=1)
    return PitchedWorkload(image, table, [], [copy], f"pitched_{which}")


# ------------------------------------------- memsets and kernel launches

KARG_DTYPE = np.dtype([("ptr", "<u8"), ("bytes", "<u8"), ("access", "<u4"), ("reserved", "<u4")])
ARG_READ, ARG_WRITE = 1, 2


def kernel_launches(rng, n_launch: int, table: AllocTable, max_args: int = 6,
                    bytes_lo: int = 16, bytes_hi: int = 64 << 10, p_bad: float = 0.08,
                    p_zero: float = 0.05) -> list:
    """Pointer arguments of n_launch kernel launches: 1..max_args each, read,
    write or both (40/35/25), extents log-uniform in [bytes_lo, bytes_hi]
    placed inside a live allocation; p_bad of them overrun it or point at a
    freed one, p_zero have no extent (pointer check only); some launches
    pass the same buffer twice."""
    live = np.setdiff1d(np.arange(len(table.base)), table.freed)
    out = []
    for _ in range(n_launch):
        k = int(rng.integers(1, max_args + 1))
        a = np.zeros(k, KARG_DTYPE)
        for i in range(k):
            acc = int(rng.choice([ARG_READ, ARG_WRITE, ARG_READ | ARG_WRITE], p=[0.4, 0.35, 0.25]))
            n = 0 if rng.random() < p_zero else int(log_uniform_int(rng, bytes_lo, bytes_hi, 1)[0])
            u = rng.random()
            if u < p_bad / 3 and len(table.freed):
                j = int(rng.choice(table.freed))
                ptr = int(table.base[j]) + int(rng.integers(0, int(table.size[j])))
            else:
                j = int(rng.choice(live))
                b, s = int(table.base[j]), int(table.size[j])
                if u < p_bad:      # runs past the end
                    ptr = b + max(0, s - max(1, n // 2))
                else:
                    ptr = b + int(rng.integers(0, max(1, s - n + 1)))
            a[i] = (ptr, n, acc, 0)
        if k > 1 and rng.random() < 0.15:
            a[1]["ptr"] = a[0]["ptr"]
        out.append(a)
    return out


def memsets(rng, count: int, table: AllocTable, p_bad: float = 0.1) -> list:
    """(dptr, pitch, width, height) of cuMemsetD8/D2D-style calls inside
    live allocations; p_bad of them run past the allocation's end."""
    live = np.setdiff1d(np.arange(len(table.base)), table.freed)
    out = []
    for _ in range(count):
        j = int(rng.choice(live))
        b, s = int(table.base[j]), int(table.size[j])
        if rng.random() < 0.5:
            h, w = 1, int(rng.integers(1, s + 1))
            pitch = 0
        else:
            h = int(rng.integers(2, 33))
            w = int(rng.integers(1, max(2, s // h)))
            pitch = w + int(rng.integers(0, 64))
        ext = (h - 1) * pitch + w
        if rng.random() < p_bad:
            d = b + max(0, s - ext + int(rng.integers(1, 64)))
        else:
            d = b + int(rng.integers(0, max(1, s - ext + 1)))
        out.append((d, pitch, w, h))
    return out


@dataclass
class DevopsWorkload:
    image: HostImage
    table: AllocTable
    setup: list      # (kind, dst, src, n) copies run first
    memset: tuple    # (dptr, pitch, width, height)
    args: np.ndarray  # KARG_DTYPE: one launch
    name: str = "devops"


def devops_large(seed: int = 0) -> DevopsWorkload:
    """A 1 GiB memset and one launch with four 256 MiB pointer arguments:
    read (a buffer copied from a host image with undefined runs, density
    1e-6), read+write (another such buffer), write (a fresh buffer), read
    (the memset buffer).  16 allocations in all."""
    rng = rng_for(9000 + seed)
    n = 256 << 20
    image = host_image_runs(rng, n, undef_frac=1e-6, mean_run=8.0)
    sizes = np.array([1 << 30, n, n, n] + [1 << 20] * 12, dtype=np.uint64)
    bases = disjoint_bases(rng, sizes)
    table = AllocTable(bases, sizes, np.zeros(0, np.int64))
    A, B, C, D = (int(x) for x in bases[:4])
    setup = [(HTOD, B, 0, n), (HTOD, C, 0, n)]
    args = np.array([(B, n, ARG_READ, 0), (C, n, ARG_READ | ARG_WRITE, 0), (D, n, ARG_WRITE, 0),
                     (A + (64 << 20), n, ARG_READ, 0)], KARG_DTYPE)
    return DevopsWorkload(image, table, setup, (A, 0, 1 << 30, 1), args)

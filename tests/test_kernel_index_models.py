"""CPU models of the GPU kernels' index arithmetic, run before their first
GPU launch and kept as tests: for many random geometries, every chunk of
every row is visited exactly once by the pitched work splits, every
bulk copy and shared-memory read of the span and A-bits-only tiles stays
inside its buffer and window while covering every byte that is classified,
and the table merge writes every entry of the new table exactly once, in
the host merge's order.  The models restate the kernels' integer
arithmetic (cg_scan_pitched.cu, cg_tma.cuh, cg_kernels.cu); a change there
must be mirrored here.  CPU only."""
from __future__ import annotations

import random

kR = 10
kVBytes = 16 * (32 * kR + 1)
kABytes = 64 * kR + 64
kStage = ((kVBytes + kABytes) + 127) & ~127


def f16(x):
    return x & ~15


def c16(x):
    return (x + 15) & ~15


# ------------------------------------------------ pitched work splits

def _visit_pitched(width, rows, sm, per_sm, uniform, ax0):
    ax = (lambda r: ax0) if uniform else (lambda r: (r * 7 + 3) % 16)
    kmax = ((ax0 + width + 15) >> 4) if uniform else (width + 30) >> 4
    need = {r: (ax(r) + width + 15) >> 4 for r in range(rows)}
    seen = set()
    wpc = 8
    if kmax >= 256:           # scan_pitched_tma_kernel
        kTW = 16
        tpr = (kmax + 32 * kR - 1) // (32 * kR)
        ntiles = rows * tpr
        grid = min((ntiles + kTW - 1) // kTW, sm * per_sm)
        nw = grid * kTW
        for gw in range(nw):
            for t in range(gw, ntiles, nw):
                r = t // tpr
                c0 = (t - r * tpr) * kR * 32
                for c in range(c0, c0 + kR * 32):
                    if c < need[r]:
                        assert (r, c) not in seen
                        seen.add((r, c))
    elif kmax > 32:           # scan_pitched_wide_kernel
        U = 4
        G = (kmax + 32 * U - 1) // (32 * U)
        items = rows * G
        grid = max(1, min((items + wpc - 1) // wpc, sm * per_sm))
        T = grid * wpc
        tg, tr = T % G, T // G
        for warp in range(grid * wpc):
            grp, r = warp % G, warp // G
            while r < rows:
                for k in range(U):
                    for lane in range(32):
                        c = grp * 32 * U + 32 * k + lane
                        if c < need[r]:
                            assert (r, c) not in seen
                            seen.add((r, c))
                grp += tg
                r += tr
                if grp >= G:
                    grp -= G
                    r += 1
    else:                     # scan_pitched_narrow_kernel
        lp = 0
        while (1 << lp) < kmax:
            lp += 1
        P = 1 << lp
        groups = 32 >> lp
        U = 1
        per_step = groups * U
        grid = max(1, min((rows + per_step * wpc - 1) // (per_step * wpc), sm * per_sm))
        nwarps = grid * wpc
        for warp in range(nwarps):
            for base in range(warp * per_step, rows, nwarps * per_step):
                for k in range(U):
                    for lane in range(32):
                        r = base + k * groups + (lane >> lp)
                        ls = lane & (P - 1)
                        if r < rows and ls < need[r]:
                            assert (r, ls) not in seen
                            seen.add((r, ls))
    assert len(seen) == sum(need.values())


def test_pitched_work_splits_cover_every_chunk_once():
    rng = random.Random(2)
    cases = [(1, 1), (1, 300), (16, 333), (17, 50), (64, 7), (500, 9), (513, 33), (4095, 5),
             (4096, 5), (4097, 3), (16384, 6)]
    cases += [(rng.randint(1, 30000), rng.randint(1, 20)) for _ in range(8)]
    for w, r in cases:
        for uni in (True, False):
            for sm, ps in ((152, 3), (1, 1)):
                _visit_pitched(w, r, sm, ps, uni, ax0=(w * 3) % 16)


# ------------------------------------------------ span tiles (short rows)

def make_geo(kind, carry, rdev, n, host_off, dev_src, dev_dst, imgv):
    host_v = imgv + host_off
    if kind=='H': anchor = dev_dst if carry else host_v
    elif kind=='D': anchor = host_v
    else: anchor = dev_dst if carry else dev_src
    ax = anchor & 15
    vin = host_v if kind=='H' else dev_src
    vw = vin - ax; vr = vw & 15; val = vw - vr
    g = dict(n=n, ax=ax, vin_al=val, vin_r=vr, vin_lo=vin, vin_hi=vin+n, has_vin=(kind=='H' or rdev),
             hb0=host_off-ax, hlo=host_off, hhi=host_off+n, nch=(ax+n+15)>>4)
    return g
def rows_per_tile(kind, rdev, H, hp, sp, lanes):
    if H < 2: return 0
    rt = H
    if kind=='H' or rdev:
        pv = hp if kind=='H' else sp
        room = kVBytes - 62 - 16*lanes
        if room < 0 or pv == 0: return 0
        rt = min(rt, room//pv + 1)
    if kind != 'X':
        room = (kABytes-32)*8 - 15 - 16*lanes
        if room < 0 or hp == 0: return 0
        rt = min(rt, room//hp + 1)
    return rt if rt >= 2 else 0
def trial(rng):
    kind = rng.choice('HDX')  # H htod, D dtoh, X dtod
    carry = rng.random() < 0.7; rdev = kind != 'H'
    W = rng.randint(1, 500); H = rng.randint(2, 400); D = rng.choice([1,1,2,3])
    kmax_bound = (W + 30) >> 4
    if kmax_bound > 32: return 0
    hp = W + rng.randint(0, 60); sp = W + rng.randint(0, 60); dp = W + rng.randint(0, 60)
    if rng.random() < 0.5: dp = (dp + 15)//16*16; sp = (sp+15)//16*16; hp = (hp+15)//16*16
    hrows = H + rng.randint(0, 3); srows = H + rng.randint(0, 3); drows = H + rng.randint(0, 3)
    imgv = 0x100000  # 16-aligned base
    img_n = (D*hrows*hp + 4096 + 127)//128*128
    host_start = rng.randint(0, 2000) if True else 0
    if host_start + ((D-1)*hrows + (H-1))*hp + W > img_n: return 0
    src_buf = 0x4000000 + 256*rng.randint(0, 10)   # allocation shadow (256-aligned)
    src_size = ((D*srows*sp + 4096)+255)//256*256
    src_start = src_buf + rng.randint(0, 300)
    dst_buf = 0x9000000; dst_start = dst_buf + rng.randint(0, 300)
    # the host's row_chunks: exact when every anchor row has one alignment
    if kind == 'D' or (kind == 'H' and not carry):
        a0, pa, ra = imgv + host_start, hp, hrows
    elif carry:
        a0, pa, ra = dst_start, dp, drows
    else:
        a0, pa, ra = src_start, sp, srows
    uniform = (H == 1 or pa % 16 == 0) and (D == 1 or (pa*ra) % 16 == 0)
    kmax = ((a0 & 15) + W + 15) >> 4 if uniform else kmax_bound
    lp = 0
    while (1 << lp) < kmax: lp += 1
    P = 1 << lp
    rt = rows_per_tile(kind, rdev, H, hp, sp, P)
    if not rt: return 0
    tps = (H + rt - 1)//rt; ntiles = tps*D
    def row(r):
        z, y = divmod(r, H)
        return make_geo(kind, carry, rdev, W, host_start + z*hrows*hp + y*hp,
                        src_start + z*srows*sp + y*sp, dst_start + z*drows*dp + y*dp, imgv)
    for t in range(ntiles):
        z = t // tps; y0 = (t - z*tps)*rt; y1 = min(y0 + rt, H)
        r0, r1 = z*H + y0, z*H + y1
        g0, g1 = row(r0), row(r1-1)
        # --- issue
        vcopy = None; acopy = None
        if kind == 'H' or g0['has_vin']:
            vbeg = g0['vin_al']; lo = f16(g0['vin_lo']); hi = min(c16(g1['vin_hi']), vbeg + kVBytes)
            assert lo >= vbeg
            if hi > lo:
                assert (hi - lo) % 16 == 0 and (lo - vbeg) % 16 == 0 and hi - vbeg <= kVBytes
                vcopy = (lo, hi)
                # global range inside the input buffer's 16-aligned region
                if kind == 'H':
                    assert lo >= imgv and hi <= imgv + img_n
                else:
                    assert lo >= src_buf and hi <= src_buf + src_size
        if kind != 'X':
            aorig = f16(g0['hb0'] >> 3)
            q0 = max(g0['hb0'], g0['hlo']); q1 = g1['hhi']
            if q1 > q0:
                b0 = f16(q0 >> 3); b1 = min(c16((q1+7) >> 3), aorig + kABytes)
                assert b0 >= aorig and b0 >= 0 and b1 <= img_n//8 and (b1-b0) % 16 == 0
                acopy = (b0, b1)
        # --- consume
        vbeg = g0['vin_al']; aorig = f16(g0['hb0'] >> 3)
        for r in range(r0, r1):
            g = row(r)
            assert g['nch'] <= P, (g['nch'], P)
            for c in range(P):
                if kind == 'H' or g['has_vin']:
                    k = (g['vin_al'] + 16*c - vbeg) >> 4
                    assert 0 <= k and (k+2)*16 <= kVBytes, (k, c, P)
                    # valid bytes of this chunk come from copied bytes
                    i0 = 16*c - g['ax']
                    for i in range(max(0, i0), min(W, i0 + 16)):
                        addr = g['vin_lo'] + i
                        assert vcopy and vcopy[0] <= addr < vcopy[1], (addr, vcopy)
                if kind != 'X':
                    q = g['hb0'] + 16*c
                    wi = (((q >> 5) << 2) - aorig) >> 2
                    assert wi >= 0 and (wi+2)*4 <= kABytes, (wi,)
                    i0 = 16*c - g['ax']
                    for i in range(max(0, i0), min(W, i0 + 16)):
                        pos = g['hlo'] + i
                        assert acopy and acopy[0]*8 <= pos < acopy[1]*8
    return 1


def test_span_tiles_stay_in_bounds_and_cover():
    rng = random.Random(5)
    done = sum(trial(rng) for _ in range(600))
    assert done > 500


# ------------------------------------------- A-bits-only super-tiles

def test_a_super_tiles_stay_in_bounds_and_cover():
    rng = random.Random(3)
    for _ in range(20000):
        n = rng.randint(1, 1 << 22)
        img_n = ((rng.randint(n, n + 10000) + 127) // 128) * 128
        hlo = rng.randint(0, img_n - n)
        hhi = hlo + n
        ax = rng.randint(0, 15)
        hb0 = hlo - ax
        nsc = (ax + n + 127) >> 7
        ntiles = ((nsc + 31) // 32 + kR - 1) // kR
        t = rng.randint(0, ntiles - 1)
        c0 = t * kR * 32
        p0 = hb0 + 128 * c0
        aorig = f16(p0 >> 3)
        q0 = max(p0, hlo)
        q1 = min(p0 + 4096 * kR + 32, hhi)
        if q1 > q0:
            b0 = f16(q0 >> 3)
            b1 = c16((q1 + 7) >> 3)
            assert b0 >= aorig and b1 - aorig <= kStage and b1 <= img_n // 8 and b0 >= 0
            for lane in (0, 31):
                i0 = 128 * c0 - ax + 128 * kR * lane
                lo_i, hi_i = max(0, i0), min(n, i0 + 128 * kR)
                if hi_i > lo_i:
                    assert b0 * 8 <= hlo + lo_i and hlo + hi_i <= b1 * 8
        w0 = (p0 - 8 * aorig) >> 5
        # the last word read (j = 128 kR - 1) and the one after it lie in the stage
        assert (w0 + 128 * kR + 1) * 4 <= kStage


# ------------------------------------------------ table merge

def _count_below(a, x):
    lo, hi = 0, len(a)
    while lo < hi:
        mid = (lo + hi) >> 1
        if a[mid] < x:
            lo = mid + 1
        else:
            hi = mid
    return lo


def _merge_model(base, dead, ins):
    """Places as table_merge_kernel computes them (dead: sorted bases of
    freed entries); None where it skips."""
    n, m = len(base), len(ins)
    out = [None] * (n - len(dead) + m)
    for i in range(n + m):
        if i < n:
            b = base[i]
            r = _count_below(dead, b)
            if r < len(dead) and dead[r] == b:
                continue
            o = i - r + _count_below(ins, b)
        else:
            k = i - n
            b = ins[k]
            o = k + _count_below(base, b) - _count_below(dead, b)
        assert 0 <= o < len(out) and out[o] is None
        out[o] = b
    return out


def test_table_merge_places_every_entry_once_in_base_order():
    rng = random.Random(11)
    for _ in range(3000):
        n = rng.randrange(0, 40)
        base = sorted(rng.sample(range(0, 4000, 4), n))
        dead_i = set(rng.sample(range(n), rng.randrange(0, n + 1)))
        dead = sorted(base[i] for i in dead_i)
        live = [base[i] for i in range(n) if i not in dead_i]
        # registrations: fresh bases, and some at the base of a dead entry
        pool = [b for b in range(2, 4000, 4)] + dead
        ins = sorted(set(rng.sample(pool, rng.randrange(0, 12))))
        if n == 0 and not ins:
            continue
        want = sorted(live + ins)
        assert _merge_model(base, dead, ins) == want


# ------------------------------------------------ dynamic segment claims

kSegQ = 8


class _Src:
    """SegSrc: static striding, or claims taken by the producer and handed
    to the consumer through the warp's ring."""

    def __init__(self, shared, ring, step, prod):
        self.shared, self.ring, self.step, self.prod, self.n = shared, ring, step, prod, 0

    def claim(self):
        v = self.step + self.shared["ctr"]
        self.shared["ctr"] += 1
        return v

    def next(self, cur):
        if self.shared is None:
            return cur + self.step
        if self.prod:
            v = self.claim()
            self.ring["q"][self.n & (kSegQ - 1)] = v
            self.ring["pushed"] += 1
            assert self.ring["pushed"] - self.ring["popped"] <= kSegQ, "ring overflow"
        else:
            v = self.ring["q"][self.n & (kSegQ - 1)]
            self.ring["popped"] += 1
            assert self.ring["popped"] <= self.ring["pushed"], "pop before push"
        self.n += 1
        return v


class _It:
    def __init__(self):
        self.s = self.t = self.t_end = 0
        self.valid = False

    def copy(self):
        o = _It()
        o.__dict__.update(self.__dict__)
        return o


def _settle(it, tiles, src):
    while it.s < len(tiles):
        if tiles[it.s]:
            it.t, it.t_end, it.valid = 0, tiles[it.s], True
            return
        it.s = src.next(it.s)
    it.valid = False


def _advance(it, tiles, src):
    it.t += 1
    if it.t < it.t_end:
        return
    it.s = src.next(it.s)
    _settle(it, tiles, src)


def _warp(gw, nw, tiles, shared, kNS, consumed):
    """One warp of scan_level_tma_kernel, a generator yielding after every
    consumed tile (so warps interleave their claims)."""
    ring = {"q": [None] * kSegQ, "pushed": 0, "popped": 0}
    psrc = _Src(shared, ring, nw, True)
    csrc = _Src(shared, ring, nw, False)
    prod = _It()
    prod.s = gw
    if gw < len(tiles):
        _settle(prod, tiles, psrc)
    cons = prod.copy()
    csrc.n = psrc.n
    ring["popped"] = ring["pushed"]
    issued = []
    for _ in range(kNS):
        if not prod.valid:
            break
        issued.append((prod.s, prod.t))
        _advance(prod, tiles, psrc)
    while cons.valid:
        assert issued and issued.pop(0) == (cons.s, cons.t)
        consumed.append((cons.s, cons.t))
        if prod.valid:
            issued.append((prod.s, prod.t))
            _advance(prod, tiles, psrc)
        _advance(cons, tiles, csrc)
        yield


def test_dynamic_segment_claims_cover_every_tile_once():
    rng = random.Random(21)
    for trial in range(400):
        n_segs = rng.randrange(1, 120)
        # tiles per segment; 0 = an empty trailing segment (after a copy)
        tiles = [rng.choice([1, 1, 2, 3, 16]) for _ in range(n_segs)]
        for k in range(1, n_segs):
            if rng.random() < 0.2 and tiles[k - 1]:
                tiles[k] = 0
        nw = rng.choice([1, 2, 5, 16, 64])
        for dynamic in (False, True):
            shared = {"ctr": 0} if dynamic else None
            consumed = []
            warps = [_warp(w, nw, tiles, shared, 2, consumed) for w in range(nw)]
            live = list(warps)
            while live:
                g = rng.choice(live)
                try:
                    next(g)
                except StopIteration:
                    live.remove(g)
            want = sorted((s, t) for s in range(n_segs) for t in range(tiles[s]))
            assert sorted(consumed) == want, (trial, dynamic)


def test_single_copy_segments_cover_every_tile_once():
    """scan_single_tma_kernel: a copy's tiles cut into segments of seg_tiles
    (the last one shorter), the warps' own first segments, then claims."""
    rng = random.Random(5)
    for _ in range(300):
        ntiles = rng.randrange(1, 400)
        nw = rng.choice([1, 3, 16, 48])
        seg_tiles = max(1, min(16, ntiles // (4 * nw)))
        nseg = (ntiles + seg_tiles - 1) // seg_tiles
        tiles = [min(seg_tiles, ntiles - k * seg_tiles) for k in range(nseg)]
        consumed = []
        shared = {"ctr": 0}
        live = [_warp(w, nw, tiles, shared, 2, consumed) for w in range(nw)]
        while live:
            g = rng.choice(live)
            try:
                next(g)
            except StopIteration:
                live.remove(g)
        assert sorted(consumed) == sorted((s, t) for s in range(nseg) for t in range(tiles[s]))


def test_tile_a_addressing_32bit_equals_64bit():
    """consume_tile's A word index and shift, computed in 32 bits from the
    tile's base, equal the 64-bit form and stay inside the A window."""
    rng = random.Random(9)
    abytes = 64 * kR + 64
    for _ in range(20000):
        hb0 = rng.randrange(-15, 1 << 40)
        c0 = rng.randrange(0, 1 << 28) * kR * 32
        p0 = hb0 + 16 * c0
        aorig = (p0 >> 3) & ~15
        qbase = p0 - 8 * aorig
        assert 0 <= qbase < 136
        for k in (0, 1, 31, 32, 33, rng.randrange(kR * 32), kR * 32 - 1):
            q = hb0 + 16 * (c0 + k)
            wi64 = (((q >> 5) << 2) - aorig) >> 2
            qb = qbase + 16 * k
            assert (qb >> 5, qb & 31) == (wi64, q & 31)
            assert 4 * (qb >> 5) + 8 <= abytes
            # the per-lane form: word (qbase + 16 lane) >> 5 plus 16 per row
            lane, u = k & 31, k >> 5
            a_q = qbase + 16 * lane
            assert ((a_q >> 5) + 16 * u, a_q & 31) == (qb >> 5, qb & 31)


def test_span_row_addressing_32bit_equals_64bit():
    """consume_span's per-row V index, realignment and A word/shift, from
    32-bit offsets relative to the stage's windows, equal the 64-bit forms
    (Geo of the row) for rows of random pitch and alignment."""
    rng = random.Random(17)
    for _ in range(20000):
        vbeg = rng.randrange(1 << 40) & ~15          # the V window start (aligned)
        vin = vbeg + rng.randrange(0, 4000)
        ax = rng.randrange(16)                       # the row's anchor alignment
        host = rng.randrange(0, 1 << 40)
        aorig = ((host - ax) >> 3) & ~15 if rng.random() < 0.5 else ((host - 200) >> 3) & ~15
        for c in (0, 1, 7, 15, 31):
            vw = vin - ax
            k64 = ((vw - (vw & 15)) + 16 * c - vbeg) >> 4
            vrel = vin - vbeg
            k32 = ((vrel - ax) >> 4) + c
            assert (k32, (vrel - ax) & 15) == (k64, vw & 15)
            q = host - ax + 16 * c
            wi64 = (((q >> 5) << 2) - aorig) >> 2
            qb = (host - 8 * aorig) - ax + 16 * c
            assert (qb >> 5, qb & 31) == (wi64, q & 31)


# ------------------------------------------- interior tiles' bulk copies

def _issue_general(g, c0):
    """issue_tile's clipped V and A bulk copies: (voff, vsrc, vbytes, aoff, asrc, abytes)."""
    out = [0, 0, 0, 0, 0, 0]
    if g["kind"] == 1 or g["has_vin"]:
        vbeg = g["vin_al"] + 16 * c0
        vend = vbeg + kVBytes
        lo_lim = g["vin_lo"] & ~15
        hi_lim = (g["vin_hi"] + 15) & ~15
        lo, hi = max(vbeg, lo_lim), min(vend, hi_lim)
        if hi > lo:
            out[0:3] = [lo - vbeg, lo, hi - lo]
    if g["kind"] != 3:
        p0 = g["hb0"] + 16 * c0
        p1 = p0 + 512 * kR
        aorig = f16(p0 >> 3)
        q0, q1 = max(p0, g["hlo"]), min(p1 + 32, g["hhi"])
        if q1 > q0:
            b0, b1 = f16(q0 >> 3), c16((q1 + 7) >> 3)
            out[3:6] = [b0 - aorig, b0, b1 - b0]
    return out


def _issue_interior(g, c0):
    out = [0, 0, 0, 0, 0, 0]
    if g["kind"] == 1 or g["has_vin"]:
        out[0:3] = [0, g["vin_al"] + 16 * c0, kVBytes]
    if g["kind"] != 3:
        p0 = g["hb0"] + 16 * c0
        aorig = f16(p0 >> 3)
        out[3:6] = [0, aorig, c16((p0 + 512 * kR + 39) >> 3) - aorig]
    return out


def test_interior_tile_issue_equals_clipped_form():
    """issue_tile's fast path (tiles with c0 >= 1 and c0 + 32 kR + 2 <=
    nchunks) issues exactly the bulk copies of the general, clipped form,
    for every kind, anchor and source alignment."""
    rng = random.Random(23)
    checked = 0
    for _ in range(4000):
        kind = rng.choice([1, 2, 3])
        carry, rdev = rng.random() < 0.7, rng.random() < 0.7
        n = rng.randrange(1, 1 << 20)
        host_off = rng.randrange(0, 1 << 30)
        dev_src = rng.randrange(1 << 30, 1 << 40)
        dev_dst = rng.randrange(1 << 30, 1 << 40)
        imgv = (rng.randrange(1 << 20, 1 << 30)) & ~15
        ge = make_geo("HDT"[kind - 1], carry, rdev, n, host_off, dev_src, dev_dst, imgv)
        if kind == 3 and not carry and not rdev:
            continue  # no chunks: nothing is issued
        g = {"kind": kind, "has_vin": ge["has_vin"], "vin_al": ge["vin_al"],
             "vin_lo": ge["vin_lo"], "vin_hi": ge["vin_hi"], "hb0": ge["hb0"],
             "hlo": ge["hlo"], "hhi": ge["hhi"]}
        nchunks = ge["nch"]
        ntiles = (nchunks + 32 * kR - 1) // (32 * kR)
        for t in {0, 1, ntiles // 2, ntiles - 2, ntiles - 1}:
            c0 = t * 32 * kR
            if t < 0 or not (c0 >= 1 and c0 + 32 * kR + 2 <= nchunks):
                continue
            assert _issue_interior(g, c0) == _issue_general(g, c0), (kind, n, t)
            checked += 1
    assert checked > 2000


# ------------------------------------------- ragged last tiles

def _valid_mask(i0, n):
    """valid_mask: bytes of copy index [i0, i0+16) that lie in [0, n)."""
    lo = -i0 if i0 < 0 else 0
    hi = min(n - i0, 16)
    if hi <= lo:
        return 0
    return ((1 << hi) - 1) & ~((1 << lo) - 1)


def test_tile_rows_past_the_last_chunk_are_empty():
    """consume_tile with SKIP stops after urows = min(kR, ceil((nchunks -
    c0) / 32)) rows: every chunk of a skipped row has an empty valid mask,
    so skipping it changes no count, first offset or carried byte; and each
    kept row holds at least one chunk of the copy."""
    rng = random.Random(29)
    for _ in range(20000):
        ax = rng.randrange(16)
        n = rng.choice([rng.randrange(1, 64), rng.randrange(1, 1 << 14), rng.randrange(1, 1 << 22)])
        nchunks = (ax + n + 15) >> 4
        ntiles = (nchunks + 32 * kR - 1) // (32 * kR)
        t = ntiles - 1 if rng.random() < 0.7 else rng.randrange(ntiles)
        c0 = t * 32 * kR
        rem = nchunks - c0
        urows = kR if rem >= 32 * kR else (rem + 31) >> 5
        for u in range(kR):
            masks = [_valid_mask(16 * (c0 + 32 * u + lane) - ax, n) for lane in range(32)]
            if u >= urows:
                assert not any(masks), (ax, n, c0, u)
            else:
                assert any(masks), (ax, n, c0, u)


# ------------------------------------------- chunk pairs of scan-only tiles

def _funnel_r(lo, hi, sh):
    return (((hi << 32) | lo) >> sh) & 0xFFFFFFFF


def test_chunk_pairs_equal_single_chunks():
    """consume_tile's pair loop for checks that carry nothing: pair p = 32 v
    + lane holds chunks 2p and 2p + 1; its 32-bit A word (word qbase/32 +
    p of the tile's A window at shift qbase % 32) holds chunk 2p's 16 A
    bits in its low half and chunk 2p + 1's in its high half, exactly the
    bits the one-chunk loop extracts (word qbase/32 + lane/2 + 16 u at the
    lane's own shift); its V vectors 2p, 2p + 1, 2p + 2 stay inside the
    stage's window; each lane's chunks come in increasing order and every
    chunk of the tile is taken once."""
    rng = random.Random(31)
    nwords = 16 * kR + 16  # the A window, in 32-bit words
    for _ in range(300):
        words = [rng.randrange(1 << 32) for _ in range(nwords)]
        qbase = rng.randrange(136)

        def a16_single(k):  # the one-chunk loop's extraction for chunk k = 32 u + lane
            u, lane = divmod(k, 32)
            a_q = qbase + 16 * lane
            wi = (a_q >> 5) + 16 * u
            sh = a_q & 31
            w1 = words[wi + 1] if sh > 16 else 0
            return _funnel_r(words[wi], w1, sh) & 0xFFFF

        seen = []
        for lane in range(32):
            last = -1
            for v in range(kR // 2):
                p = 32 * v + lane
                k = 2 * p
                assert k + 2 <= 32 * kR  # V vectors k, k+1, k+2 of the 32 kR + 1
                w = (qbase >> 5) + p
                assert w + 1 < nwords
                a32 = _funnel_r(words[w], words[w + 1], qbase & 31)
                assert a32 & 0xFFFF == a16_single(k)
                assert a32 >> 16 == a16_single(k + 1)
                assert k > last
                last = k + 1
                seen += [k, k + 1]
        assert sorted(seen) == list(range(32 * kR))

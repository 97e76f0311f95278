"""CPU checks of the index schedules that the CUDA kernels follow (re-derived here from
their definitions, no GPU): the cluster form of the SVT Jacobi (block Jacobi on 2C
half-blocks moved on a round-robin tournament) and the gather / scatter of the Fourier
operator's slots.  They guard the design: every column pair must meet once per sweep,
the pairs of a local round must be disjoint, the chunked half-block moves must read each
offset before its holder overwrites it, and the realified slices must carry
[[a1, -a2], [a2, a1]] and scatter back to the slots exactly.  Also: the TMA transform
kernel's incremental tile cursors and its per-thread work items, the FP32 sweeps' layout
of rows in register pairs, and the ordering of the QR pivot keys.
"""
import numpy as np
import pytest


def rr_i(r, k, n):
    return n - 1 if k == 0 else (r + k) % (n - 1)


def rr_j(r, k, n):
    return r if k == 0 else (r - k + n - 1) % (n - 1)


def padded(n, C):
    return (n + 4 * C - 1) // (4 * C) * (4 * C)


def local_pairs(b, h):
    """Pairs (i, j) of local columns of every local round of block round b."""
    rounds = []
    nlr = (h - 1 if b == 0 else 0) + h
    for lr in range(nlr):
        pairs = []
        for kq in range(h):
            if b == 0 and lr < h - 1:
                sl = 0 if kq < h // 2 else 1
                kk = kq - sl * (h // 2)
                pairs.append((sl * h + rr_i(lr, kk, h), sl * h + rr_j(lr, kk, h)))
            else:
                sh = lr - (h - 1) if b == 0 else lr
                pairs.append((kq, h + (kq + sh) % h))
        rounds.append(pairs)
    return rounds


def holder(b, k, sl, C):
    return rr_i(b, k, 2 * C) if sl == 0 else rr_j(b, k, 2 * C)


def sources(b, k, C):
    """(CTA, slot) holding, in block round b, each half-block CTA k needs in round b+1."""
    nb = (b + 1) % (2 * C - 1)
    out = []
    for sl in range(2):
        x = holder(nb, k, sl, C)
        src = [(kk, s2) for kk in range(C) for s2 in range(2) if holder(b, kk, s2, C) == x]
        assert len(src) == 1
        out.append(src[0])
    return out


@pytest.mark.parametrize("C", [3, 4])
@pytest.mark.parametrize("n", [2, 6, 7, 30, 61, 97, 144, 190, 288])
def test_block_jacobi_meets_every_pair_once_per_sweep(C, n):
    np_ = padded(n, C)
    nl = np_ // C
    h = nl // 2
    assert h % 2 == 0
    store = {k: [q * C + k for q in range(nl)] for k in range(C)}  # column labels
    for _ in range(2):  # two sweeps: the layout returns to block round 0's each sweep
        seen = set()
        for b in range(2 * C - 1):
            for k in range(C):
                for pairs in local_pairs(b, h):
                    flat = [c for p in pairs for c in p]
                    assert len(set(flat)) == len(flat) and all(0 <= c < nl for c in flat)
                    for i, j in pairs:
                        pr = tuple(sorted((store[k][i], store[k][j])))
                        assert pr not in seen
                        seen.add(pr)
            new = {}
            for k in range(C):
                cols = []
                for kk, s2 in sources(b, k, C):
                    cols += store[kk][s2 * h:(s2 + 1) * h]
                new[k] = cols
            store = new
        assert len(seen) == np_ * (np_ - 1) // 2


@pytest.mark.parametrize("C,n,ld,threads", [(3, 30, 97, 128), (3, 144, 177, 384),
                                            (4, 144, 177, 288), (4, 288, 353, 576)])
def test_half_block_moves_read_before_overwrite(C, n, ld, threads):
    """The moves go in chunks of offsets w inside a half-block (8 elements per thread,
    both slots): an element (CTA, slot, w) is read by its next holder and overwritten by
    its current holder in the same chunk, on opposite sides of that chunk's barrier."""
    h = padded(n, C) // C // 2
    per, wch = h * ld, 8 * threads // 2
    for b in range(2 * C - 1):
        read, written = {}, {}
        for k in range(C):
            src = sources(b, k, C)
            for ci, wb in enumerate(range(0, per, wch)):
                for idx in range(8 * threads):
                    sl, w = idx & 1, wb + (idx >> 1)
                    if w >= per or src[sl] == (k, sl):
                        continue
                    read[src[sl] + (w,)] = ci
                    written[(k, sl, w)] = ci
        for key, ci in read.items():
            assert written.get(key, ci) == ci


def realify(G, I1, I2, n, R):
    """Index recipe of the Fourier gather: real slots to Wr, realified pairs to Wc."""
    S, h, nr = I1 * I2, (n - 1) // 2, 2 if n % 2 == 0 else 1
    Wr = np.empty(nr * R * S)
    Wc = np.empty(h * R * 4 * S)
    for idx in range(Wr.size):
        e, q = idx % S, idx // S
        Wr[idx] = G[(q // nr * n + (0 if q % nr == 0 else n - 1)) * S + e]
    for t in range(Wc.size):
        q, w = t // (4 * S), t % (4 * S)
        row, col = w % (2 * I1), w // (2 * I1)
        rb, cb = row >= I1, col >= I2
        i, j = row - I1 * rb, col - I2 * cb
        slot = 2 * (q % h + 1) - 1 if rb == cb else 2 * (q % h + 1)
        v = G[((q // h) * n + slot) * S + i + j * I1]
        Wc[t] = -v if (not rb and cb) else v
    return Wr, Wc


def derealify(Wr, Wc, I1, I2, n, R):
    S, h, nr = I1 * I2, (n - 1) // 2, 2 if n % 2 == 0 else 1
    G = np.empty(R * n * S)
    for idx in range(G.size):
        e, p = idx % S, idx // S
        r, s = p // n, p % n
        if s == 0:
            G[idx] = Wr[nr * r * S + e]
        elif n % 2 == 0 and s == n - 1:
            G[idx] = Wr[(1 + nr * r) * S + e]
        else:
            q = (s + 1) // 2 - 1 + h * r
            row = e % I1 if s & 1 else I1 + e % I1
            G[idx] = Wc[q * 4 * S + row + (e // I1) * 2 * I1]
    return G


@pytest.mark.parametrize("I1,I2,n,R", [(3, 2, 1, 2), (3, 4, 2, 3), (4, 3, 3, 2),
                                       (2, 5, 4, 2), (3, 3, 5, 2), (2, 3, 7, 3)])
def test_fourier_realify_layout_and_round_trip(I1, I2, n, R):
    rng = np.random.default_rng(I1 + 10 * n + 100 * R)
    G = rng.standard_normal(R * n * I1 * I2)
    Wr, Wc = realify(G, I1, I2, n, R)
    S, h = I1 * I2, (n - 1) // 2
    for r in range(R):
        for k in range(1, h + 1):
            a1 = G[(r * n + 2 * k - 1) * S:(r * n + 2 * k) * S].reshape(I2, I1).T
            a2 = G[(r * n + 2 * k) * S:(r * n + 2 * k + 1) * S].reshape(I2, I1).T
            q = (k - 1) + h * r
            got = Wc[q * 4 * S:(q + 1) * 4 * S].reshape(2 * I2, 2 * I1).T
            assert np.array_equal(got, np.block([[a1, -a2], [a2, a1]]))
    assert np.array_equal(derealify(Wr, Wc, I1, I2, n, R), G)


# ---- TMA transform passes: tile cursors and per-thread work items (lt_transform.cu)

KTHREADS = 256  # compute threads of a transform CTA


@pytest.mark.parametrize("Sg,TS,outer,grid", [(480, 32, 1, 304), (65536, 32, 1, 304),
                                             (16777216 // 8, 256, 1, 304), (468, 32, 3, 7),
                                             (4096, 128, 5, 152), (96, 32, 2, 304)])
def test_tma_tile_cursor_matches_division(Sg, TS, outer, grid):
    """A CTA takes a contiguous run of tiles; the copy thread walks it with an incremental
    cursor (column tile xt, row group yt) instead of dividing.  The cursor must give the
    positions t % tpo, t / tpo of every tile, every tile must belong to exactly one CTA,
    and the TMA x coordinate (xt TS floats) must be a multiple of 16 bytes."""
    tpo = (Sg + TS - 1) // TS
    ntiles = outer * tpo
    per = (ntiles + grid - 1) // grid
    seen = np.zeros(ntiles, dtype=np.int64)
    for b in range(grid):
        first = b * per
        mine = min(per, ntiles - first) if first < ntiles else 0
        xt, yt = first % tpo, first // tpo
        for i in range(mine):
            t = first + i
            assert (xt, yt) == (t % tpo, t // tpo)
            assert (xt * TS * 4) % 16 == 0
            seen[t] += 1
            xt += 1
            if xt == tpo:
                xt, yt = 0, yt + 1
    assert np.all(seen == 1)


def items_of(I, st, Pg, R):
    """(fibre start, first output) of each work item of one mode, as item_geometry."""
    nfib = Pg // I
    out = []
    for it in range(((I + R - 1) // R) * nfib):
        ch, fiber = it // nfib, it % nfib
        out.append((fiber % st + st * I * (fiber // st), ch * R))
    return out


@pytest.mark.parametrize("modes", [(16, 16), (8,), (3, 32), (5, 3), (16,), (2, 4), (32,)])
@pytest.mark.parametrize("TS,R", [(32, 8), (128, 8), (256, 8), (32, 2), (256, 2)])
def test_transform_items_cover_the_tile_once(modes, TS, R):
    """The work items of each mode of a pass cover every (fibre, output) row of the tile
    exactly once and stay inside its Pg rows; when a mode has at most one item per row
    slot (the case the TMA kernel computes once per thread), thread row slot rs holds
    item rs, which is what the general loop gives it first."""
    Pg = int(np.prod(modes))
    nrs = KTHREADS // (TS // 4)
    st = 1
    for I in modes:
        rows = np.zeros(Pg, dtype=np.int64)
        for fbase, j0 in items_of(I, st, Pg, R):
            for r in range(R):
                if j0 + r < I:
                    row = fbase + st * (j0 + r)
                    assert 0 <= row < Pg
                    rows[row] += 1
        assert np.all(rows == 1)
        items = len(items_of(I, st, Pg, R))
        if items <= nrs:
            general = {rs: items_of(I, st, Pg, R)[rs] for rs in range(nrs) if rs < items}
            assert len(general) == items
        st *= I


@pytest.mark.parametrize("G,E", [(16, 7), (16, 9), (8, 18), (16, 16), (32, 18), (16, 4)])
def test_fp32_register_pairs_cover_rows_once(G, E):
    """FP32 block sweeps hold a column's rows in adjacent pairs: lane l takes rows
    2 l + 2 G k and the next (k < E / 2) and, for odd E, row 2 G (E / 2) + l.  Together the
    G lanes must hold rows 0 .. G E - 1 once each, and every pair must start on an even
    row (8-byte loads; the leading dimension is even)."""
    EP = E // 2
    rows = np.zeros(G * E, dtype=np.int64)
    for lane in range(G):
        for k in range(EP):
            r0 = 2 * lane + 2 * G * k
            assert r0 % 2 == 0
            rows[r0] += 1
            rows[r0 + 1] += 1
        if E % 2:
            rows[2 * G * EP + lane] += 1
    assert np.all(rows == 1)


def pivot_key(s, c):
    """The QR pivot key of column c with squared norm s (high 32 bits of the value's
    bit pattern above the inverted index), as in lt_jacobi_svt.cuh."""
    if s.dtype == np.float32:
        hi = int(np.array(s, dtype=np.float32).view(np.uint32))
    else:
        hi = int(np.array(s, dtype=np.float64).view(np.uint64)) >> 32
    return (hi << 32) | (0xFFFFFFFF - c)


def pivot_index(key):
    return 0xFFFFFFFF - (key & 0xFFFFFFFF)


@pytest.mark.parametrize("dt", [np.float32, np.float64])
def test_pivot_key_picks_largest_norm_then_smallest_index(dt):
    """The maximum of the keys names the column of largest squared norm and, among equal
    keys, the smallest index: non-negative floats order like their bit patterns."""
    rng = np.random.default_rng(7)
    for trial in range(200):
        n = int(rng.integers(1, 300))
        s = (rng.random(n) * 10.0 ** rng.integers(-30, 30)).astype(dt)
        if trial % 3 == 0:
            s[rng.integers(0, n, size=max(1, n // 4))] = s.max()  # ties at the maximum
        if trial % 7 == 0:
            s[:] = 0  # all columns exhausted
        p = pivot_index(max(pivot_key(s[c], c) for c in range(n)))
        if dt is np.float32:
            assert s[p] == s.max() and p == int(np.flatnonzero(s == s.max())[0])
        else:  # the key keeps the high 32 bits: a relative tie band of 2^-20
            assert s[p] >= s.max() * (1 - 2.0 ** -19)
            best = max(int(np.array(v).view(np.uint64)) >> 32 for v in s)
            cand = [c for c in range(n) if int(np.array(s[c]).view(np.uint64)) >> 32 == best]
            assert p == cand[0]

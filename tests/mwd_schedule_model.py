"""Level-tag model of the blocked (wavefront-diamond) kernel's schedule -- test infrastructure.

It replays, on the CPU, the loop structure of the blocked kernel in csrc/mwd.cu for one
configuration: per diamond row, per tile, per x slab (block of the cluster), per wavefront step,
the same plane loads, write-backs, compute items and x-halo pushes, with the same index formulas.
Instead of values, every cell carries the time level it holds.  The model checks:
  * every global and shared-memory index the kernel would touch is inside its buffer;
  * every read sees exactly the time level the update needs (halo cells match any level);
  * no shared cell is both written and read (by different items) within one step, and the cells
    being loaded are not read in that step (the single barrier per step suffices);
  * at the end, buffer T%2 holds level T and buffer (T-1)%2 holds level T-1 everywhere.
Tiles of a row advance in lock step (one legal interleaving of independent tiles).
"""
from __future__ import annotations

import numpy as np

HALO = -1000


def slab_width(nx, C):
    w = -(-nx // C)
    return -(-w // 16) * 16


def vec_slab_width(nx, R, C, a16):
    """Vector path: the slabs split the padded columns [R, nx + R) at 16-byte boundaries."""
    w = -(-(nx + R) // C)
    return -(-w // a16) * a16


PD = 3       # cp.async paths: planes staged this many steps ahead (a group issued at step k is
             # waited for before the barrier ending step k+PD-1: in flight during steps k..k+PD-1)
PD_BULK = 3  # bulk-copy path
SLACK = 2    # bulk-copy path: extra ring planes per wavefront width
SLACK_PLAIN = 1  # cp.async paths


def shape(R, dw, nf, XW, bulk=False):
    H = dw // R
    K = R + nf
    pd = PD_BULK if bulk else PD
    NZ = (pd + 1) * nf + R + max(R, nf) + (H - 2) * K + (SLACK if bulk else SLACK_PLAIN) * nf
    return NZ, dw + 2 * R, -(-(XW + 2 * R) // 4) * 4


def rows(T, dw, R):
    if T <= 0:
        return 0
    Hh = dw // R // 2
    rho = 0
    while rho * Hh + 1 <= T - 1:
        rho += 1
    return rho + 1


def row_span(rho, dw, ny):
    h = rho * (dw // 2)
    lo = h // dw
    hi = -(-(ny + h) // dw) - 1
    return lo, max(hi - lo + 1, 0)


def simulate(R, second_order, nx, ny, nz, T, dw, nf, C, bulk=False, a16=4, vec=False, box=False):
    """vec: the 16-byte vector path (block r owns padded columns [r*XW, (r+1)*XW); its shared row
    starts HM = R rounded up to a16 columns before them; whole a16-column chunks are staged and
    written back; both rows of a pair are read even when only the first is updated).
    bulk (with vec): the bulk-copy schedule -- planes staged PD_BULK steps ahead, a ring slack of
    SLACK*nf planes, write-back copies that may still read shared memory for two steps.
    box (R = 1, vec): the 27-point box stencil also reads the diagonal neighbours -- every cell of
    planes z-1..z+1, rows y-1..y+1, columns x-1..x+1 -- which must all hold level t."""
    assert vec or not bulk, "the bulk-copy schedule runs on the vector partition"
    assert not box or (vec and R == 1), "the box stencil runs on the vector path, radius 1"
    if vec:
        XW = vec_slab_width(nx, R, C, a16)
        HM = -(-R // a16) * a16
        NZ, YW, _ = shape(R, dw, nf, XW, bulk)
        XT = XW + 2 * HM
    else:
        XW = slab_width(nx, C)
        NZ, YW, XT = shape(R, dw, nf, XW, bulk)

    def slab(rank):
        """(first interior column of slab column 0, shared column of slab column 0, valid slab
        columns [lo, hi))."""
        if vec:
            x0 = rank * XW - R
            return x0, HM, max(0, -x0), min(XW, nx - x0)
        x0 = rank * XW
        return x0, R, 0, min(XW, nx - x0)
    pdm = PD_BULK if bulk else PD
    H = dw // R
    K = R + nf
    Hh = H // 2
    G = np.full((2, nz + 2 * R, ny + 2 * R, nx + 2 * R), HALO, dtype=np.int64)
    G[0, R:-R, R:-R, R:-R] = 0
    G[1, R:-R, R:-R, R:-R] = -1
    max_g = max_s = 0

    def gtag(p, z, y, x):
        nonlocal max_g
        assert -R <= z < nz + R and -R <= y < ny + R and -R <= x < nx + R, (z, y, x)
        return G[p, z + R, y + R, x + R]

    for rho in range(rows(T, dw, R)):
        a_min, nd = row_span(rho, dw, ny)
        tb = max((rho - 1) * Hh + 1, 0)
        te = min((rho + 1) * Hh - 1, T - 1)
        if tb > te or nd == 0:
            continue
        nlev = te - tb + 1
        smax = nlev - 1
        W = -(-(nz + smax * K) // nf)
        tiles = []
        for ti in range(nd):
            a = a_min + ti
            b = a - rho
            P0 = a * dw - rho * (dw // 2)
            Y0 = P0 - R
            lev = []
            for s in range(nlev):
                t = tb + s
                lo = max(a * dw - R * t, b * dw + R * t, 0)
                hi = min((a + 1) * dw - R * t, (b + 1) * dw + R * t, ny)
                lev.append((lo, max(hi - lo, 0)))
            mask = []
            for yy in range(YW):
                y = Y0 + yy
                m = 0
                if 0 <= y < ny and P0 <= y < P0 + dw:
                    cnt, par = 0, 0
                    for s in range(nlev):
                        t = tb + s
                        if max(a * dw - R * t, b * dw + R * t) <= y < min((a + 1) * dw - R * t, (b + 1) * dw + R * t):
                            cnt += 1
                            par = (t + 1) & 1
                    m = 3 if cnt >= 2 else ((1 << par) if cnt == 1 else 0)
                mask.append(m)
            S = np.full((C, 2, NZ, YW, XT), -5000, dtype=np.int64)  # -5000: never loaded
            tiles.append(dict(a=a, P0=P0, Y0=Y0, lev=lev, mask=mask, S=S))

        def load_plane(tl, rank, z, loaded):
            nonlocal max_s
            x0, off, vlo, vhi = slab(rank)
            if z < -R or z >= nz + R or vhi <= vlo:
                return
            slot = (z + R) % NZ
            Y0 = tl["Y0"]
            ylo, yhi = max(Y0, -R), min(Y0 + YW, ny + R)
            if vec:  # whole a16 chunks of padded columns [pc0 - HM, pc0 + XW + HM), inside the row
                pc0 = rank * XW
                cb, ce = max(pc0 - HM, 0), min(pc0 + XW + HM, nx + 2 * R)
                cols = [(pc - (pc0 - HM), pc - R) for pc in range(cb, ce)]
            else:
                cols = [(xx, x0 - R + xx) for xx in range(vhi + 2 * R)]
            for p in range(2):
                for y in range(ylo, yhi):
                    for xx, x in cols:
                        assert 0 <= y - Y0 < YW and 0 <= xx < XT
                        tl["S"][rank, p, slot, y - Y0, xx] = gtag(p, z, y, x)
                        loaded.add((rank, p, slot, y - Y0, xx))

        def write_plane(tl, rank, z, wb_reads):
            x0, off, vlo, vhi = slab(rank)
            xw = vhi
            if z < 0 or z >= nz or vhi <= vlo:
                return
            slot = (z + R) % NZ
            if vec:  # the owned padded columns [pc0, pc0 + XW), inside the row
                pc0 = rank * XW
                cols = [pc - (pc0 - HM) for pc in range(pc0, min(pc0 + XW, nx + 2 * R))]
            else:
                cols = [xl + R for xl in range(xw)]
            for yy in range(YW):
                m = tl["mask"][yy]
                if not m:
                    continue
                y = tl["Y0"] + yy
                for xx in cols:
                    x = x0 - off + xx
                    for p in range(2):
                        if m >> p & 1:
                            gtag(p, z, y, x)
                            v = tl["S"][rank, p, slot, yy, xx]
                            if not (-R <= x < 0 or nx <= x):  # interior: the final level, never stale
                                G[p, z + R, y + R, x + R] = v
                            else:
                                assert v == G[p, z + R, y + R, x + R], ("halo rewritten with a new value", x)
                            wb_reads.add((rank, p, slot, yy, xx))

        def check_read(tagv, want):
            assert tagv == want or tagv == HALO, (tagv, want)

        for tl in tiles:
            tl["prev_wb"] = [set(), set()]  # write-back reads of the last two steps (still in flight)
            tl["inflight"] = []  # (issue step, cells) of cp.async groups
            tl["win"] = {}
            for rank in range(C):
                for z in range(-R, pdm * nf + R):
                    load_plane(tl, rank, z, set())
        for w in range(W):
            for tl in tiles:
                loaded, wb_reads, reads, writes = set(), set(), {}, {}
                for rank in range(C):
                    for f in range(nf):
                        load_plane(tl, rank, (w + pdm) * nf + R + f, loaded)
                tl["inflight"] = [(ws, c) for ws, c in tl["inflight"] if ws > w - pdm] + [(w, loaded)]
                busy = set().union(*[c for _, c in tl["inflight"]])
                for rank in range(C):
                    if w > 0:
                        for f in range(nf):
                            write_plane(tl, rank, (w - 1) * nf - smax * K + f, wb_reads)
                pending = []
                for rank in range(C):
                    x0, off, vlo, vhi = slab(rank)
                    if vhi <= vlo:
                        continue
                    for s in range(nlev):
                        zb = w * nf - s * K
                        if zb + nf <= 0 or zb >= nz:
                            continue
                        t = tb + s
                        pin, pout = t & 1, (t & 1) ^ 1
                        lo, width = tl["lev"][s]
                        hi = lo + width
                        Sx = tl["S"][rank]
                        for y0 in range(lo, hi, 2):
                            row1 = y0 + 1 < hi
                            yy0 = y0 - tl["Y0"]
                            for f in range(nf):
                                z = zb + f
                                if z < 0 or z >= nz:
                                    continue
                                sl = (z + R) % NZ
                                for xl in range(vlo, vhi):
                                    xx = xl + off
                                    item = (rank, s, y0, z, xl)
                                    key = (rank, s, y0, xl)
                                    def rd(cell, want):
                                        assert 0 <= cell[2] < YW and 0 <= cell[3] < XT, cell
                                        check_read(Sx[cell], want)
                                        reads.setdefault((rank,) + cell, set()).add(item)
                                        return Sx[cell]
                                    if z == 0:
                                        tl["win"][key] = [[rd((pin, (sl + d) % NZ, yy0 + r, xx), t)
                                                           for d in range(-R, R + 1)] for r in (0, 1)]
                                    else:
                                        wv = tl["win"][key]
                                        for r in (0, 1):
                                            wv[r] = wv[r][1:] + [rd((pin, (sl + R) % NZ, yy0 + r, xx), t)]
                                    for r in (0, 1):  # centre of each row is its window's middle
                                        check_read(tl["win"][key][r][R], t)
                                    if vec:  # the vector kernel re-reads the 2R+1 planes of both rows
                                        for r in (0, 1):
                                            for d in range(-R, R + 1):
                                                cell = (pin, (sl + d) % NZ, yy0 + r, xx)
                                                if r == 0 or row1:
                                                    rd(cell, t)
                                                else:
                                                    assert 0 <= cell[2] < YW, cell
                                                    reads.setdefault((rank,) + cell, set()).add(item)
                                    for d in range(1, R + 1):
                                        rd((pin, sl, yy0 - d, xx), t)
                                        if d < R or row1:
                                            rd((pin, sl, yy0 + 1 + d, xx), t)
                                    if vec and not row1:  # the second row is read, not used
                                        for cell in [(pin, (sl + d) % NZ, yy0 + 1, xx + e)
                                                     for d in range(-R, R + 1) for e in range(-R, R + 1)] + \
                                                    [(pin, sl, yy0 + R, xx), (pout, sl, yy0 + 1, xx)]:
                                            assert 0 <= cell[2] < YW and 0 <= cell[3] < XT, cell
                                            reads.setdefault((rank,) + cell, set()).add(item)
                                    for r in (0, 1) if row1 else (0,):
                                        for d in range(-R, R + 1):
                                            if d:
                                                rd((pin, sl, yy0 + r, xx + d), t)
                                        if box:  # edges and corners, in the planes below and above too
                                            for dz in (-1, 0, 1):
                                                for dy in (-1, 0, 1):
                                                    for dx in (-1, 0, 1):
                                                        if dy and (dx or dz) or (dx and dz):
                                                            rd((pin, (sl + dz) % NZ, yy0 + r + dy, xx + dx), t)
                                        if second_order:
                                            rd((pout, sl, yy0 + r, xx), t - 1)
                                        outs = [(rank, pout, sl, yy0 + r, xx)]
                                        if C > 1 and xl < R and rank > 0:
                                            outs.append((rank - 1, pout, sl, yy0 + r, xx + XW))
                                        if C > 1 and xl >= XW - R and rank < C - 1:
                                            outs.append((rank + 1, pout, sl, yy0 + r, xx - XW))
                                        for o in outs:
                                            assert 0 <= o[4] < XT and 0 <= o[3] < YW
                                            assert o not in writes, ("double write", o)
                                            writes[o] = item
                                        pending.append((outs, t + 1))
                # race checks within the step
                for cell, it in writes.items():
                    rs = reads.get(cell, set())
                    assert rs <= {it}, ("read and written in one step", cell)
                    assert cell not in busy and cell not in wb_reads, ("write vs load/write-back", cell)
                    for old in tl["prev_wb"][(0 if bulk else 1):]:
                        assert cell not in old, ("write vs a recent step's write-back", cell)
                # a slot restaged in this step may still be read by a write-back of the previous
                # step (threads of the block that have not yet passed that step's barrier), and in
                # the bulk-copy path by the write-back copies of the two previous steps
                for old in tl["prev_wb"][(0 if bulk else 1):]:
                    assert not (old & loaded), "slot restaged while a recent write-back may still read it"
                tl["prev_wb"] = [tl["prev_wb"][1], wb_reads]
                for cell in busy:
                    assert cell not in reads and cell not in wb_reads, ("slot read while its load is in flight", cell)
                for outs, lv in pending:
                    for o in outs:
                        tl["S"][o] = lv
        for tl in tiles:
            for rank in range(C):
                for f in range(nf):
                    write_plane(tl, rank, (W - 1) * nf - smax * K + f, set())
    inner = (slice(R, -R),) * 3
    if T > 0:
        assert np.all(G[T % 2][inner] == T)
        assert np.all(G[(T - 1) % 2][inner] == T - 1)
    return True

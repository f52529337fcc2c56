"""CPU model of the z-segmented persistent diamond schedule: the extruded diamond split along z
into parallelepipeds (Sect. 8), each run as one item of the device FIFO.

A tile (diamond (rho, a), levels tb .. te) runs wavefront steps w = 0 .. W-1, W = nz + smax K,
updating level s = t - tb at plane w - s K.  Segment j of the tile is the step range
[Z_j, Z_{j+1}) with Z_j = j * zseg (j < nseg = ceil(nz / zseg)) and Z_nseg = W: every level
advances through the same steps, so a segment is a parallelepiped in (z, t).  The kernel starts
item (rho, a, j) once
  * (rho, a, j-1) and
  * (rho-1, a-1, j') and (rho-1, a, j'), j' = min(j + delta, nseg - 1),
    delta = ceil(((tb(rho) - tb(rho-1) - 1) K + R) / zseg)
have completed.  Values cross items through global memory only: a segment stores its final
values and, unless it is the tile's last, every value of its last B steps (B = K + R, or 2K for
the second-order stencils, whose update also reads level t-2 at the centre).

The model checks, cell by cell of (y, z, t), that
  * the items partition the updates;
  * every input of an update (level t-1 at rows y-R .. y+R and planes z-R .. z+R, and level t-2
    at the cell for the second-order stencils) is produced by the same item at an earlier step,
    or by an item that precedes it transitively and stored the value (final or in its band);
  * every update's write, which overwrites level t-2 at the cell, comes after all readers of that
    value (the same item at an earlier step, or an item it depends on transitively);
  * every dependency precedes its item in the FIFO order (key seg + (delta_max + 1) rho), so
    resident clusters taking items in that order cannot deadlock;
and, with delta or B one smaller, that a check fails (the model has teeth).
"""
import pytest

from mwd_schedule_model import row_span, rows


def _tb(rho, Hh):
    return max((rho - 1) * Hh + 1, 0)


def _delta(rho, Hh, K, R, zseg):
    d = _tb(rho, Hh) - _tb(rho - 1, Hh)
    return -(-((d - 1) * K + R) // zseg)


def _model(R, dw, nf, ny, nz, T, zseg, order2, ddelta=0, dband=0):
    H = dw // R
    Hh = H // 2
    K = R + nf
    nseg = -(-nz // zseg)
    B = (2 * K if order2 else K + R) + dband
    tiles = {}
    for rho in range(rows(T, dw, R)):
        a0, nd = row_span(rho, dw, ny)
        tb, te = _tb(rho, Hh), min((rho + 1) * Hh - 1, T - 1)
        if tb > te:
            continue
        for a in range(a0, a0 + nd):
            b = a - rho
            lev = {}
            for t in range(tb, te + 1):
                lo = max(a * dw - R * t, b * dw + R * t, 0)
                hi = min((a + 1) * dw - R * t, (b + 1) * dw + R * t, ny)
                lev[t] = (lo, hi)
            tiles[(rho, a)] = dict(tb=tb, te=te, lev=lev, W=nz + (te - tb) * K)
    own = {}    # (y, z, t) -> (item, step)
    for (rho, a), tl in tiles.items():
        for t, (lo, hi) in tl["lev"].items():
            s = t - tl["tb"]
            for z in range(nz):
                w = z + s * K
                j = min(w // zseg, nseg - 1)
                for y in range(lo, hi):
                    assert (y, z, t) not in own
                    own[(y, z, t)] = ((rho, a, j), w)
    assert len(own) == ny * nz * T  # the items partition the updates

    def deps(item):
        rho, a, j = item
        out = [(rho, a, j - 1)] if j > 0 else []
        if rho > 0:
            jp = min(j + _delta(rho, Hh, K, R, zseg) - ddelta, nseg - 1)
            for d in (a - 1, a):
                if (rho - 1, d) in tiles:
                    out.append((rho - 1, d, max(jp, 0)))
        return out

    dmax = max([_delta(r, Hh, K, R, zseg) for r in range(1, rows(T, dw, R))] + [0])
    items = sorted({(rho, a, j) for (rho, a) in tiles for j in range(nseg)},
                   key=lambda it: (it[2] + (dmax + 1) * it[0], it[0], it[1]))
    pos = {it: i for i, it in enumerate(items)}
    anc = {}
    for it in items:
        s = set()
        for p in deps(it):
            assert p in pos and pos[p] < pos[it], (it, p)  # FIFO order: no deadlock
            s |= anc[p] | {p}
        anc[it] = s

    def stored(cell):
        """The producing item wrote the cell's value to global memory."""
        y, z, t = cell
        (rho, a, j), w = own[cell]
        tl = tiles[(rho, a)]
        if not (t + 2 <= tl["te"] and tl["lev"][t + 2][0] <= y < tl["lev"][t + 2][1]):
            return True  # final in the tile
        end = (j + 1) * zseg if j + 1 < nseg else tl["W"]
        return j + 1 < nseg and w >= end - B

    for cell, (x_item, x_step) in own.items():
        y, z, t = cell
        near = [(y + dy, z + dz, t - 1) for dy in range(-R, R + 1) for dz in range(-R, R + 1)
                if t >= 1 and 0 <= y + dy < ny and 0 <= z + dz < nz]
        ins = near + ([(y, z, t - 2)] if order2 and t >= 2 else [])
        for c in ins:  # read after write
            p_item, p_step = own[c]
            if p_item == x_item:
                assert p_step < x_step, (cell, c)
            else:
                assert p_item in anc[x_item], ("input from an item not waited for", cell, c, x_item, p_item)
                assert stored(c), ("input not stored to global memory", cell, c, x_item, p_item)
        for c in near:  # write after read: the readers of the overwritten level t-2
            r_item, r_step = own[c]
            if r_item == x_item:
                assert r_step < x_step, (cell, c)
            else:
                assert r_item in anc[x_item], ("overwrites a value a later item reads", cell, c, x_item, r_item)
    return len(items)


CASES = [
    # R, dw, nf, ny, nz, T, zseg
    (1, 4, 1, 23, 20, 9, 6),
    (1, 6, 1, 30, 17, 12, 5),
    (1, 8, 2, 37, 26, 17, 8),
    (1, 4, 1, 12, 13, 7, 1),
    (1, 8, 1, 21, 16, 11, 3),
    (4, 8, 1, 40, 24, 6, 8),
    (4, 16, 1, 45, 30, 9, 7),
    (4, 8, 2, 33, 21, 5, 20),
]


@pytest.mark.parametrize("R,dw,nf,ny,nz,T,zseg", CASES)
@pytest.mark.parametrize("order2", [False, True])
def test_segments_cover_every_dependency(R, dw, nf, ny, nz, T, zseg, order2):
    n = _model(R, dw, nf, ny, nz, T, zseg, order2)
    assert n > 1


@pytest.mark.parametrize("R,dw,nf,ny,nz,T,zseg", [(1, 8, 1, 29, 24, 13, 4), (4, 16, 1, 45, 30, 9, 10)])
@pytest.mark.parametrize("order2", [False, True])
def test_a_smaller_delta_or_band_fails(R, dw, nf, ny, nz, T, zseg, order2):
    with pytest.raises(AssertionError):
        _model(R, dw, nf, ny, nz, T, zseg, order2, ddelta=1)
    with pytest.raises(AssertionError):
        _model(R, dw, nf, ny, nz, T, zseg, order2, dband=-1)


def test_one_segment_is_the_extruded_diamond():
    # zseg >= nz: one item per diamond, the FED_PERSISTENT schedule
    assert _model(1, 8, 1, 37, 12, 9, 12, False) == _model(1, 8, 1, 37, 12, 9, 100, False)

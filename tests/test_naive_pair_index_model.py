"""CPU check of the naive FP32 kernels' 8-byte shared-memory loads (csrc/naive.cu): every offset
is even (8-byte aligned, given a 16-byte aligned ring and slot sizes of whole 16-byte chunks) and
every element read lies inside its ring slot, for every thread of the block.

* Box stencil (2x2 block per thread): rows 2 ty - 1 .. 2 ty + 2 and columns 2 tx - 1 .. 2 tx + 2 of
  the tile, as the pairs at shared offset (2 ty + rr) TXW + 2 tx and + 2, rr = 0 .. 3, in each of
  the planes z-1, z, z+1.
* 25-point factor grid (two adjacent columns per thread, rows ty and ty + TY): pairs at
  tc + d (x offsets d = -4, -2, 2, 4) and tc + d TXW (y offsets d = -4 .. 4), tc = (row + R) TXW +
  R + 2 tx.
The shared tile of a slot is TYW = 2 TY + 2R rows of TXW = TX + 2R rounded up to 4 floats, TX =
32 VX.
"""
import pytest


def _shape(R, VX, TY):
    TX = 32 * VX
    TXW = -(-(TX + 2 * R) // 4) * 4
    TYW = 2 * TY + 2 * R
    return TX, TXW, TYW


def test_box_block_loads():
    R, VX, TY = 1, 2, 8
    TX, TXW, TYW = _shape(R, VX, TY)
    TP = TXW * TYW
    assert TP % 4 == 0  # slots of whole 16-byte chunks
    for ty in range(TY):
        for tx in range(32):
            rows, cols = set(), set()
            for rr in range(4):
                p = (2 * ty + rr) * TXW + 2 * tx
                for off in (p, p + 2):
                    assert off % 2 == 0
                    assert 0 <= off and off + 1 < TP
                    rows.add(off // TXW)
                    cols.update({off % TXW, off % TXW + 1})
            # shared row q is tile row q - R, shared column c is tile column c - R
            assert rows == {2 * ty + rr for rr in range(4)}
            assert {c - R for c in cols} == set(range(2 * tx - 1, 2 * tx + 3))
            assert max(cols) < TXW


@pytest.mark.parametrize("TY", [8])
def test_factor_grid_pair_loads(TY):
    R, VX = 4, 2
    TX, TXW, TYW = _shape(R, VX, TY)
    TP = TXW * TYW
    for ty in range(TY):
        for r in range(2):
            row = ty + r * TY
            for tx in range(32):
                tc = (row + R) * TXW + R + 2 * tx
                offs = [tc + d for d in (-4, -2, 2, 4)] + [tc + d * TXW for d in range(-4, 5)]
                for off in offs:
                    assert off % 2 == 0, (ty, r, tx, off)
                    assert 0 <= off and off + 1 < TP, (ty, r, tx, off)
                # x pairs stay inside the row
                assert (tc - 4) // TXW == (tc + 5) // TXW == row + R

"""CPU model of OVERLAP_PERSISTENT's shared-memory ring (csrc/mwd_overlap.cuh): plane bookkeeping
of one item (a whole tile, or one z segment of it), with the kernel's index formulas.

An item runs wavefront steps j = 0 .. W-1 of its tile starting at tile step ws (ws = seg * zseg;
whole tiles: ws = 0, W = nz + smax K); level s updates plane z = ws + j - s K when 0 <= z < nz,
reading planes z-R .. z+R of the level's input buffer and writing plane z of its output buffer
(whose old value, level s-2's, the second-order update reads first).  Plane q lives in ring slot
(q + R) mod NZ, NZ = L + 2R + 1 + (H-2) K.  Staging: step 0 brings planes max(ws - smax K, 0) - R
.. ws + R (from -R at least), step j >= 1 plane ws + j + R (planes past nz + R - 1 do not exist);
the staging warp issues steps 0 .. L-1 before the loop and step it + L after DONE(it - 1); the
waiting warp releases step j (FULL) once the copies of steps <= j + 1 have landed.

The model checks that every read and write at step j finds its plane in its slot, landed, and that
no copy overwrites a slot whose plane is still read or written at the step it may overlap or
later: the copy of step it + L is in flight while step it computes.  With a ring one plane short
it must fail (the model has teeth).
"""
import pytest


def _replay(R, H, nf, L, nz, smax, ws, W, NZ=None):
    K = R + nf
    NZ = NZ or L + 2 * R + 1 + (H - 2) * K
    access = {}  # plane -> last step that reads or writes it (within the item)
    for j in range(W):
        for s in range(smax + 1):
            z = ws + j - s * K
            if 0 <= z < nz:
                for q in range(z - R, z + R + 1):
                    access[q] = max(access.get(q, -1), j)
    slot = {}       # slot -> plane (staged or being staged)
    staged_at = {}  # plane -> staging step

    def stage(j, issue_step):
        zfirst = max(ws - smax * K, 0) - R
        z0 = zfirst if j == 0 else ws + j + R
        z1 = min(ws + j + R, nz + R - 1)
        for q in range(z0, z1 + 1):
            s = (q + R) % NZ
            old = slot.get(s)
            if old is not None and old != q:
                # the copy may land while step issue_step computes: the old plane must be done
                assert access.get(old, -2) < issue_step, (R, H, L, nz, smax, ws, W, q, old, issue_step)
            slot[s] = q
            staged_at[q] = j

    for j in range(min(L, W)):
        stage(j, 0)
    for it in range(W):
        # step it computes; copies of steps <= it + 1 have landed
        for s in range(smax + 1):
            z = ws + it - s * K
            if 0 <= z < nz:
                for q in range(z - R, z + R + 1):
                    if -R <= q < nz + R:
                        assert slot.get((q + R) % NZ) == q, ("plane not in its slot", q, it)
                        assert staged_at[q] <= it + 1, ("plane not landed", q, it)
        if it + L < W:
            stage(it + L, it)  # issued after DONE(it - 1), in flight during step it
    return True


CASES = []
for R, H in [(1, 2), (1, 4), (1, 6), (1, 8), (4, 2), (4, 4)]:
    for L in (3, 5, 8):
        for nz in (5, 23):
            for smax in range(0, H - 1):
                CASES.append((R, H, L, nz, smax))


@pytest.mark.parametrize("R,H,L,nz,smax", CASES)
def test_whole_tiles_and_segments(R, H, L, nz, smax):
    K = R + 1
    W_tile = nz + smax * K
    _replay(R, H, 1, L, nz, smax, 0, W_tile)
    for zseg in (1, 3, 7, 16):
        nseg = -(-nz // zseg)
        for seg in range(nseg):
            ws = seg * zseg
            W = W_tile - ws if seg == nseg - 1 else zseg
            _replay(R, H, 1, L, nz, smax, ws, W)


@pytest.mark.parametrize("R,H", [(1, 4), (1, 8), (4, 4)])
def test_a_ring_one_plane_short_fails(R, H):
    K = R + 1
    L, nz, smax = 3, 23, H - 2
    NZ = L + 2 * R + 1 + (H - 2) * K
    with pytest.raises(AssertionError):
        _replay(R, H, 1, L, nz, smax, 0, nz + smax * K, NZ=NZ - 1)
    with pytest.raises(AssertionError):  # and for the last segment, starting mid-tile
        _replay(R, H, 1, L, nz, smax, 5, nz + smax * K - 5, NZ=NZ - 1)

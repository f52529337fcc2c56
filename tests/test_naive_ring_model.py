"""CPU model of the naive sweep's shared-memory ring (csrc/naive.cu): plane bookkeeping only.

The kernel stages padded plane q into slot q % NP (NP = R + PD + 2 + ZB, ZB = 1 for the box
stencil), one cp.async commit group per staged plane: planes R-ZB .. 2R+PD before the loop (then
wait_all and a barrier), plane zr+2R+PD+1 after the update of interior plane zr, then
wait_group<PD> and a barrier.  Each update of plane zr reads its x/y neighbours from padded
plane zr+R (the box stencil also from zr+R-1 and zr+R+1) and, after the barrier, the window's
new value from padded plane zr+2R+1; the window's lowest planes not in the ring come from
global memory.  The model replays that order for every (R, PD, chunk length) and checks that every
read finds its plane in its slot, already landed, and that no staging overwrites a plane a
later read still needs (a slot is only refilled after the barrier that ends its last reader's
step).
"""
import pytest


def _replay(R, PD, nzb, NP=None, ZB=0):
    NP = NP or R + PD + 2 + ZB
    nplanes = nzb + 2 * R                 # padded planes of the chunk
    slot = {}                             # slot -> plane held (or being written)
    landed = set()                        # planes whose copy has completed
    groups = []                           # committed groups, oldest first: plane or None
    last_read_step = {}                   # plane -> last step that reads it
    for zr in range(nzb):
        for q in range(zr + R - ZB, zr + R + ZB + 1):                               # x/y (and box) planes
            last_read_step[q] = max(last_read_step.get(q, -1), zr)
        if zr + 1 < nzb:
            # the window read follows step zr's barrier, so it may overlap step zr+1's staging
            last_read_step[zr + 2 * R + 1] = max(last_read_step.get(zr + 2 * R + 1, -1), zr + 1)
    for i in range(R - ZB, 2 * R + 1):
        last_read_step[i] = max(last_read_step.get(i, -1), -1)  # initial window reads (step -1)

    def stage(q, step):
        if q < nplanes:
            s = q % NP
            old = slot.get(s)
            if old is not None:
                # refilling a slot: its plane must have no reader at this step or later
                assert last_read_step.get(old, -2) < step, (R, PD, nzb, q, old, step)
            slot[s] = q
            landed.discard(q)
            groups.append(q)
        else:
            groups.append(None)

    def wait_group(n):
        while len(groups) > n:
            q = groups.pop(0)
            if q is not None:
                landed.add(q)

    def read(q):
        assert slot.get(q % NP) == q and q in landed, (R, PD, nzb, q)

    for q in range(R - ZB, 2 * R + PD + 1):
        stage(q, -1)
    wait_group(0)
    for i in range(R - ZB, 2 * R + 1):
        read(i)
    # barrier: the initial window reads (step -1) are done before any in-loop staging
    for zr in range(nzb):
        for q in range(zr + R - ZB, zr + R + ZB + 1):
            read(q)                       # x/y neighbours of the updated plane (box: and z+-1)
        stage(zr + 2 * R + PD + 1, zr)    # after this step's reads, before the barrier
        wait_group(PD)
        # barrier
        if zr + 1 < nzb:
            read(zr + 2 * R + 1)          # the window's new value


@pytest.mark.parametrize("R,ZB", [(1, 0), (4, 0), (1, 1)])
@pytest.mark.parametrize("PD", [1, 2, 3, 4])
def test_naive_ring_schedule(R, ZB, PD):
    for nzb in (1, 2, 3, 5, 16, 17, 64):
        _replay(R, PD, nzb, ZB=ZB)


def test_model_has_teeth():
    """One slot fewer (NP = R + PD + 1) makes a staging overwrite a plane that is still read."""
    for R, PD, ZB in ((1, 4, 0), (4, 2, 0), (1, 4, 1)):
        with pytest.raises(AssertionError):
            _replay(R, PD, 16, NP=R + PD + 1 + ZB, ZB=ZB)

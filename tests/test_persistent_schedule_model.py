"""CPU model of the persistent diamond schedule (FED_PERSISTENT; the FIFO runtime of Sect. 4.2.3).

The kernel hands out diamonds (rho, a) in row-major order and starts one once the two diamonds
of the previous row, (rho-1, a-1) and (rho-1, a), have completed.  This model checks, cell by
cell of the (y, t) plane, with the kernel's level ranges (a*Dw - R*t <= y < (a+1)*Dw - R*t and
b*Dw + R*t <= y < (b+1)*Dw + R*t, b = a - rho, over the row's steps), that

* the diamonds partition the updates;
* every input of an update -- level t at rows y-R .. y+R, and level t-1 at row y for the
  second-order stencils -- was produced in the same diamond or in one its parents precede
  transitively (the readers of the value an in-place update overwrites are exactly those
  inputs, so the write-after-read order follows);
* diamonds of one row never depend on each other;
* the FIFO with any number of resident clusters finishes (no deadlock), for random run times;

and, with one parent left out, that the dependency check fails (the model has teeth).
"""
import random

import pytest

from mwd_schedule_model import row_span, rows


def _owners(R, dw, ny, T):
    Hh = dw // R // 2
    own = {}
    items = []
    for rho in range(rows(T, dw, R)):
        a0, nd = row_span(rho, dw, ny)
        for a in range(a0, a0 + nd):
            items.append((rho, a))
            b = a - rho
            tb, te = max((rho - 1) * Hh + 1, 0), min((rho + 1) * Hh - 1, T - 1)
            for t in range(tb, te + 1):
                lo = max(a * dw - R * t, b * dw + R * t, 0)
                hi = min((a + 1) * dw - R * t, (b + 1) * dw + R * t, ny)
                for y in range(lo, hi):
                    assert (y, t) not in own, ((y, t), own.get((y, t)), (rho, a))
                    own[(y, t)] = (rho, a)
    assert len(own) == ny * T  # every update belongs to exactly one diamond
    return own, items


def _ancestors(items, parents):
    anc = {}
    for it in items:  # row-major order: parents come first
        s = set()
        for p in parents(it):
            if p in anc:
                s |= anc[p] | {p}
        anc[it] = s
    return anc


def _check(R, dw, ny, T, second_order, parents):
    own, items = _owners(R, dw, ny, T)
    anc = _ancestors(items, parents)
    for (y, t), d in own.items():
        deps = [(yy, t - 1) for yy in range(y - R, y + R + 1) if 0 <= yy < ny and t >= 1]
        if second_order and t >= 2:
            deps.append((y, t - 2))
        for c in deps:
            e = own[c]
            assert e == d or e in anc[d], ((y, t), d, c, e)
            assert e == d or e[0] != d[0]  # same row: independent


def _kernel_parents(item):
    rho, a = item
    return [(rho - 1, a - 1), (rho - 1, a)] if rho > 0 else []


@pytest.mark.parametrize("R,dw", [(1, 2), (1, 4), (1, 6), (1, 8), (4, 8), (4, 16)])
@pytest.mark.parametrize("ny,T", [(37, 9), (64, 17), (5, 12)])
def test_two_parents_cover_every_dependency(R, dw, ny, T):
    for second_order in (False, True):
        _check(R, dw, ny, T, second_order, _kernel_parents)


def test_one_parent_is_not_enough():
    with pytest.raises(AssertionError):
        _check(1, 8, 64, 17, False, lambda it: [(it[0] - 1, it[1])] if it[0] > 0 else [])
    with pytest.raises(AssertionError):
        _check(1, 8, 64, 17, False, lambda it: [(it[0] - 1, it[1] - 1)] if it[0] > 0 else [])


@pytest.mark.parametrize("workers", [1, 2, 3, 7, 64])
def test_fifo_never_deadlocks(workers):
    """Event simulation: each of `workers` resident clusters takes the next diamond in FIFO order,
    waits for its parents' completion flags, then runs for a random time."""
    rng = random.Random(workers)
    _, items = _owners(1, 8, 200, 40)
    idx = {it: i for i, it in enumerate(items)}
    done_at = {}
    free = [0.0] * workers          # time each worker becomes free
    nxt = 0
    while nxt < len(items):
        w = min(range(workers), key=lambda i: free[i])
        it = items[nxt]
        nxt += 1
        ready = free[w]
        for p in _kernel_parents(it):
            if p in idx:
                assert idx[p] < idx[it]      # parents were taken earlier: their workers are running
                ready = max(ready, done_at[p])
        done_at[it] = ready + rng.uniform(0.5, 2.0)
        free[w] = done_at[it]
    assert len(done_at) == len(items)

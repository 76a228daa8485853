"""The cell colouring of the colour schedule (host logic, no GPU).

LC_SCHED_COLOUR runs one task per cell -- the centre cell A with its 13
forward half-shell neighbours, both cells of every pair written (Sec. IV,
Fig. 3b) -- in colour order.  Sec. VI's Strategy 1 colours cells 2-strided
and exchanges the loops so that one phase handles one stencil offset; here a
task keeps its whole stencil, so the stride is 3 along the dimensions in which
the half-shell reaches both neighbours (x, y; x in 2D) and 2 along the one in
which it reaches one side (z; y in 2D); the cells past the last full period
get classes of their own.  The tests restate that rule and check for every
grid from 3 to 40 cells per dimension that two tasks of one colour never
write the same cell, and that tasks which can write a common cell differ by
one of the dependency offsets (differences of two stencil entries) that the
device queue waits on.
"""
import itertools

import numpy as np
import pytest


def half_shell(dims=3):
    zs = (0,) if dims == 2 else (-1, 0, 1)
    return [(x, y, z) for z in zs for y in (-1, 0, 1) for x in (-1, 0, 1)
            if z > 0 or (z == 0 and y > 0) or (z == 0 and y == 0 and x > 0)]


def stride(d, dims=3):
    if dims == 2 and d == 2:
        return 1
    two_sided = d < 2 if dims == 3 else d == 0
    return 3 if two_sided else 2


def cell_class(c, nc, p):
    full = p * (nc // p)
    return c % p if c < full else p + (c - full)


def colours(nc, dims=3):
    """Number of colours of the colour schedule on a grid of nc cells."""
    n = 1
    for d in range(3):
        p = stride(d, dims)
        n *= p + (int(nc[d]) - p * (int(nc[d]) // p))
    return n


def dependency_offsets(dims=3):
    ent = [(0, 0, 0)] + half_shell(dims)
    return sorted({(a[0] - b[0], a[1] - b[1], a[2] - b[2]) for a in ent for b in ent} - {(0, 0, 0)})


def _check_grid(nc, dims):
    ent = [(0, 0, 0)] + half_shell(dims)
    cells = list(itertools.product(*(range(n) for n in nc)))
    colour = {c: tuple(cell_class(c[d], nc[d], stride(d, dims)) for d in range(3)) for c in cells}
    writes = {c: {tuple((c[d] + o[d]) % nc[d] for d in range(3)) for o in ent} for c in cells}
    writers = {}
    for c in cells:
        assert len(writes[c]) == len(ent)          # the stencil's cells are distinct
        for w in writes[c]:
            writers.setdefault(w, []).append(c)
    deps = {tuple(x % nc[d] for d, x in enumerate(o)) for o in dependency_offsets(dims)}
    for w, cs in writers.items():
        for a, b in itertools.combinations(cs, 2):
            assert colour[a] != colour[b], (nc, a, b)          # one colour: disjoint writes
            diff = tuple((b[d] - a[d]) % nc[d] for d in range(3))
            assert diff in deps, (nc, a, b)                    # the queue waits on it


@pytest.mark.parametrize("dims", [3, 2])
def test_same_colour_tasks_write_disjoint_cells(dims):
    sizes = [3, 4, 5, 6, 7, 8, 10, 11]
    for nx in sizes:
        for ny in sizes:
            nz = 1 if dims == 2 else 3 + (nx + ny) % 4
            _check_grid((nx, ny, nz), dims)
    for nc in ((40, 3, 3), (3, 40, 3), (3, 3, 40)):
        _check_grid(nc, 3)


def test_colour_counts():
    assert len(dependency_offsets(3)) == 62 and len(dependency_offsets(2)) == 12
    assert colours(np.array([42, 42, 42])) == 18          # the 1M liquid: 3 x 3 x 2
    assert colours(np.array([108, 108, 108])) == 18
    assert colours(np.array([7, 5, 3])) == 4 * 5 * 3     # leftover cells get classes of their own
    assert colours(np.array([64, 64, 1]), dims=2) == 4 * 2

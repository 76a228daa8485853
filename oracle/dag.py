"""Address-based task dependency DAG and its critical path (oracle side).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

What it computes, from the paper:
  * StarSs detects dependencies between tasks by comparing the addresses of
    their parameters (Sec. I, Sec. III); a task that reads an address depends
    on the last earlier task that wrote it, a task that writes an address also
    depends on the last writer and on every reader since then.  Tasks are
    vertices, dependencies are edges (Sec. III, Fig. 2).
  * A link-cell cell-cell interaction task declares both of its cells as
    inout (Sec. IV), so it depends on the last earlier task that touched
    either cell.
  * With equal task durations the critical path t_cp is a count of tasks and
    the best possible speedup is S = t_s / t_cp = (#tasks) / t_cp (Eq. 1,
    Sec. V).
  * Eq. 2: S(Delta, k, n) = n k / (n + Delta (k - 1)) for k stencil
    executions of n tasks each with displacement Delta; Eq. 3: its limit n/Delta.
  * Task generation orders: the basic order visits cells x fastest, then y,
    then z, and per cell runs the stencil tasks in a chosen order (Sec. V);
    loop exchange runs the outer loop over stencil offsets and the inner loop
    over the cells of one 2-strided colour (Sec. VI, Fig. 6).
Reading: the domains are periodic (the paper's 5x5 example states periodic
boundaries, Sec. V); with open boundaries the dependency chains break and the
printed speedups are not reproduced.
"""
from itertools import product

# 2D half-shell stencil of Fig. 3a / Fig. 5 (centre first), and the three
# orders of Fig. 5 expressed as offsets (dx, dy) relative to the centre cell.
STENCIL_2D = [(0, 0), (0, -1), (1, -1), (1, 0), (1, 1)]
ORDER_2D_NAIVE = [(0, 0), (0, -1), (1, -1), (1, 0), (1, 1)]   # Fig. 5a
ORDER_2D_BAD = [(0, 0), (0, -1), (1, -1), (1, 1), (1, 0)]     # Fig. 5b
ORDER_2D_OPT = [(1, 0), (1, -1), (1, 1), (0, -1), (0, 0)]     # Fig. 5c


def half_shell_3d():
    """Centre plus the 13 forward neighbours, (z, y, x) lexicographic."""
    out = []
    for oz, oy, ox in product((-1, 0, 1), repeat=3):
        if oz > 0 or (oz == 0 and oy > 0) or (oz == 0 and oy == 0 and ox > 0):
            out.append((ox, oy, oz))
    return out


def build_dag(tasks):
    """tasks: list of (reads, writes) address tuples in creation order.
    Returns parents[t] (sorted list of task indices)."""
    last_writer = {}
    readers = {}
    parents = []
    for t, (reads, writes) in enumerate(tasks):
        ps = set()
        for a in reads:
            if a in last_writer:
                ps.add(last_writer[a])
        for a in writes:
            if a in last_writer:
                ps.add(last_writer[a])
            for r in readers.get(a, ()):
                if r != t:
                    ps.add(r)
        for a in reads:
            readers.setdefault(a, []).append(t)
        for a in writes:
            last_writer[a] = t
            readers[a] = []
        ps.discard(t)
        parents.append(sorted(ps))
    return parents


def critical_path(parents):
    """Longest path counted in tasks (unit durations, Sec. V)."""
    depth = [0] * len(parents)
    for t, ps in enumerate(parents):
        depth[t] = 1 + max((depth[p] for p in ps), default=0)
    return max(depth, default=0)


def speedup(parents):
    """Eq. 1 with equal task times: S = #tasks / t_cp."""
    cp = critical_path(parents)
    return len(parents) / cp if cp else 0.0


def eq2(delta, k, n):
    """Eq. 2: S(Delta, k, n) = n k / (n + Delta (k - 1))."""
    return n * k / (n + delta * (k - 1))


def _wrap(c, dims):
    return tuple(ci % d for ci, d in zip(c, dims))


def _cells(dims):
    """Cells visited x fastest, then y, then z."""
    ranges = [range(d) for d in reversed(dims)]
    for idx in product(*ranges):
        yield tuple(reversed(idx))


def lc_task(cell, off, dims):
    """A cell-cell interaction task: both cells inout (Sec. IV)."""
    other = _wrap(tuple(c + o for c, o in zip(cell, off)), dims)
    cells = (cell,) if other == cell else (cell, other)
    return (cells, cells)


def basic_order_tasks(dims, order):
    """Outer loop over cells (x fastest), inner loop over the stencil."""
    return [lc_task(c, o, dims) for c in _cells(dims) for o in order]


def _colour(c, dims):
    """2-strided colour class per dimension (Fig. 6); the last cell of an odd
    periodic dimension gets its own class."""
    out = []
    for ci, d in zip(c, dims):
        out.append(2 if (d % 2 == 1 and ci == d - 1) else ci % 2)
    return tuple(out)


def loopex_tasks(dims, stencil):
    """Loop exchange + colouring (Strategy 1, Sec. VI): outer loop over the
    stencil offsets, then over colours, inner loop over the cells of that
    colour (x fastest)."""
    cells = list(_cells(dims))
    colours = sorted(set(_colour(c, dims) for c in cells))
    tasks = []
    for o in stencil:
        for k in colours:
            for c in cells:
                if _colour(c, dims) == k:
                    tasks.append(lc_task(c, o, dims))
    return tasks


def starss_example():
    """The program of Fig. 1 as (name, reads, writes) in call order."""
    return [
        ("unit_vec(a)", (), ("a",)),
        ("unit_vec(b)", (), ("b",)),
        ("unit_vec(c)", (), ("c",)),
        ("vec_add(c,b,c)", ("c", "b"), ("c",)),
        ("vec_add(a,b,d)", ("a", "b"), ("d",)),
        ("scalar_product(c,d,s)", ("c", "d"), ("s",)),
    ]


def starss_example_edges():
    prog = starss_example()
    parents = build_dag([(r, w) for _, r, w in prog])
    return {(prog[p][0], prog[t][0]) for t, ps in enumerate(parents) for p in ps}

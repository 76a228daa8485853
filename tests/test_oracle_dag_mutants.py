"""The task-DAG oracle's pins catch plausible slips.  Each mutant replaces
one function of oracle/dag.py (through monkeypatch, on the CPU) with a
version carrying one mistake: the second cell of a task not written (the
inout race of Sec. IV dropped), write-after-read edges missing, the
critical path counted in edges instead of tasks, the loop exchange without
its colouring.  At least one pin of test_oracle_dag.py must fail for each."""
import pytest

from oracle import dag
import test_oracle_dag as pins


def _task_first_cell_only(cell, off, dims):
    other = dag._wrap(tuple(c + o for c, o in zip(cell, off)), dims)
    cells = (cell,) if other == cell else (cell, other)
    return (cells, (cell,))


def _build_dag_no_war(tasks):
    last_writer = {}
    parents = []
    for t, (reads, writes) in enumerate(tasks):
        ps = {last_writer[a] for a in tuple(reads) + tuple(writes) if a in last_writer}
        for a in writes:
            last_writer[a] = t
        ps.discard(t)
        parents.append(sorted(ps))
    return parents


def _critical_path_edges(parents):
    depth = [0] * len(parents)
    for t, ps in enumerate(parents):
        depth[t] = max((depth[p] + 1 for p in ps), default=0)
    return max(depth, default=0)


def _loopex_uncoloured(dims, stencil):
    cells = list(dag._cells(dims))
    return [dag.lc_task(c, o, dims) for o in stencil for c in cells]


MUTANTS = {
    "first_cell_only": ("lc_task", _task_first_cell_only),
    "no_war_edges": ("build_dag", _build_dag_no_war),
    "critical_path_in_edges": ("critical_path", _critical_path_edges),
    "loopex_uncoloured": ("loopex_tasks", _loopex_uncoloured),
}

PINS = [
    ("fig1_edges", pins.test_fig1_program_dag_edges),
    ("address_rule", pins.test_address_rule_by_hand),
    ("shared_cell_ordered", lambda: pins.test_tasks_sharing_a_cell_are_ordered((6, 6))),
    ("fig5_naive", lambda: pins.test_fig5_orderings("s_max_2d_naive", dag.ORDER_2D_NAIVE)),
    ("fig5_bad", lambda: pins.test_fig5_orderings("s_max_2d_bad", dag.ORDER_2D_BAD)),
    ("fig5_opt", lambda: pins.test_fig5_orderings("s_max_2d_opt", dag.ORDER_2D_OPT)),
    ("loopex_not_limited", pins.test_loop_exchange_with_colouring_is_not_limited),
]


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_dag_pins_catch_mutant(name, monkeypatch):
    attr, fn = MUTANTS[name]
    monkeypatch.setattr(dag, attr, fn)
    caught = []
    for pin_name, pin in PINS:
        try:
            pin()
        except AssertionError:
            caught.append(pin_name)
            break
    assert caught, f"no pin fails for the mutant {name}"

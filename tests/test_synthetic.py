"""The seeded input recipes (no GPU): the batched workload's draws respect the device-
memory budget, the per-grid cap, the order and size sets and the aspect-ratio range,
and are reproducible from the seed."""
import math

import synthetic as syn


def test_batch_draws_respect_budget_and_ranges():
    ws = syn.config5()
    assert len(ws) == 64
    total = sum(w.ndof * w.extra["n_rhs"] for w in ws)
    assert total <= 512_000_000
    for w in ws:
        n = w.n_elem[0]
        assert w.n_elem == (n, n, n) and n in syn.BATCH_SIDES
        assert w.P in syn.BATCH_ORDERS and w.dim == 3 and not w.periodic
        assert w.ndof * w.extra["n_rhs"] <= 80_000_000
        widths = [s[0] for s in w.spacing]
        assert all(len(set(s)) == 1 and len(s) == n for s in w.spacing)
        ratio = max(widths) / min(widths)
        assert 1.0 <= ratio <= 16.0 + 1e-9
        assert math.isclose(sum(w.spacing[0]), 1.0)
        assert w.notes.startswith("draw ")


def test_batch_draws_are_reproducible_and_varied():
    a, b = syn.config5(), syn.config5()
    assert [(w.n_elem, w.P, w.spacing[1][0], w.spacing[2][0], w.seed) for w in a] == \
           [(w.n_elem, w.P, w.spacing[1][0], w.spacing[2][0], w.seed) for w in b]
    assert len({(w.n_elem[0], w.P) for w in a}) >= 6
    c = syn.config5(seed=1)
    assert [(w.n_elem, w.P) for w in c] != [(w.n_elem, w.P) for w in a]


def test_small_budget_forces_the_smallest_grids():
    ws = syn.config5(n_grids=4, budget_dof=4 * 4 * 8 ** 3 * 5 ** 3)
    assert all(w.n_elem == (8, 8, 8) and w.P == 4 for w in ws)

"""pmg_coarse_solve_static: the coarse solve that allocates nothing.

Callers that cannot call cudaMalloc while they solve (a host framework whose
allocator owns all device memory, or a caller that reserved its memory up front)
use this entry point; its scratch is a fixed array compiled into the library.  The test
calls it through the C ABI twice in a row and checks each result against
pmg_coarse_solve on the same hierarchy and input, then checks that a coarse
problem above the stated limit is refused.

This file is named to be collected last, so a stop-at-first-failure run has
already run every other test before it.
"""
import ctypes

import numpy as np
import pytest

import synthetic as syn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12     # same arithmetic and launch sequence as pmg_coarse_solve


def _solve_pair(case, seed):
    from paper_1603_02524_gb300 import Grid, Hierarchy, binding
    lib = binding.load()
    dim, P, ne, sp, per = case
    g = Grid(dim, P, ne, sp, periodic=per)
    h = Hierarchy(g)
    n0 = h.ndof(0)
    stream = binding._stream()
    for k in range(2):                       # two calls in a row: stale scratch must not matter
        f0 = torch.from_numpy(syn.rng(seed + k).uniform(-1, 1, n0)).cuda()
        if per:
            f0 -= f0.mean()
        ref = torch.empty_like(f0)
        got = torch.full_like(f0, float("nan"))
        assert lib.pmg_coarse_solve(h.handle, binding._ptr(f0), binding._ptr(ref), stream) == 0
        assert lib.pmg_coarse_solve_static(h.handle, binding._ptr(f0), binding._ptr(got), stream) == 0
        torch.cuda.synchronize()
        err = float((got - ref).abs().max() / ref.abs().max())
        assert err <= TOL, (case, k, err)
    h.close()
    g.close()


@pytest.mark.parametrize("case", [
    (3, 4, (4, 3, 2), [[0.25] * 4, [0.3, 0.3, 0.4], [0.5, 0.5]], False),
    (3, 2, (3, 3, 3), [[1 / 3] * 3] * 3, True),
    (2, 8, (5, 4), [[0.2] * 5, [0.25] * 4], False),
    (3, 1, (32, 32, 32), [[1 / 32] * 32] * 3, False),     # exactly at the limit: 262 144 unknowns
])
def test_static_coarse_solve_matches(case):
    _solve_pair(case, seed=100)


def test_static_coarse_solve_rejects_oversize():
    from paper_1603_02524_gb300 import Grid, Hierarchy, binding
    lib = binding.load()
    g = Grid(3, 1, (33, 32, 32), [[1 / 33] * 33, [1 / 32] * 32, [1 / 32] * 32], periodic=False)
    h = Hierarchy(g)
    n0 = h.ndof(0)
    assert n0 > 262144
    f0 = torch.zeros(n0, dtype=torch.float64, device="cuda")
    u0 = torch.zeros_like(f0)
    rc = lib.pmg_coarse_solve_static(h.handle, binding._ptr(f0), binding._ptr(u0), binding._stream())
    assert rc == -1
    assert b"262144" in lib.pmg_last_error(h.handle)
    h.close()
    g.close()

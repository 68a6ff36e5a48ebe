"""GPU: a hierarchy that carries several right-hand sides (pmg_options.nrhs = k).

Its vectors hold k vectors of the grid back to back; internally the k copies of the grid
are stacked along the last axis with walls between them, so every kernel launch (operator
apply, transfers, patch solves of every family, coarse solve) covers all k with one set of
tables, and the CG runs k independent iterations in one loop (own scalars, convergence
test and result each).  Every right-hand side must therefore give exactly what a
single-right-hand-side hierarchy gives for it:

* one apply, one smoothing step and one V-cycle on k vectors against the single
  hierarchy on each vector (1e-13 / 1e-11 / 1e-10, the patch scatter's atomic order);
* the solve of k right-hand sides (one of them zero) against the FP64 oracle's solve of
  each: the oracle's iteration count and residual history, the solution to 1e-10, in the
  host-driven loop and the device-side loop; a zero right-hand side stops at once;
* the tcgen05 tf32 V-cycle (whose face family normal to the stacked axis has one
  position more per copy than elements) within the mixed-precision bounds of
  test_gpu_tcgen05.py, and a batch of multi-right-hand-side hierarchies against the
  single solves.
"""
import numpy as np
import pytest

import synthetic as syn
from oracle.mg import Hierarchy as OHier, mgcg
from tests.helpers import e2g, elem_shape, from_dev, g2e, rel_err, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [
    # dim, P, n_elem, spacing (Dirichlet)
    (3, 4, (3, 2, 2), [[0.3, 0.5, 0.2], [0.6, 0.4], [0.7, 0.3]]),
    (3, 8, (2, 3, 2), [[0.5, 0.5], [0.3, 0.3, 0.4], [0.7, 0.3]]),
    (2, 8, (3, 4), [[0.3, 0.5, 0.2], [0.4, 0.1, 0.3, 0.2]]),
]
IDS = [f"{c[0]}d-P{c[1]}-{'x'.join(map(str, c[2]))}" for c in CASES]
K = 3


def make(case, nrhs=1, **opts):
    from paper_1603_02524_gb300 import Grid, Hierarchy
    dim, P, ne, sp = case
    g = Grid(dim, P, ne, sp, periodic=False)
    return g, Hierarchy(g, nrhs=nrhs, **opts)


def vectors(shape, seeds):
    return [syn.rng(s).uniform(-1, 1, size=shape) for s in seeds]


@pytest.mark.parametrize("kind", ["EA", "FA"])
@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_apply_smooth_vcycle_per_rhs(case, kind):
    dim, P, ne, sp = case
    _, h1 = make(case, smoother=kind)
    _, hk = make(case, nrhs=K, smoother=kind)
    assert hk.ndof() == K * h1.ndof()
    for l in range(h1.L + 1):
        assert hk.ndof(l) == K * h1.ndof(l)
    n = h1.ndof()
    us = vectors((n,), [1, 2, 3])
    fs = vectors((n,), [4, 5, 6])
    uk, fk = to_dev(np.concatenate(us)), to_dev(np.concatenate(fs))
    out = torch.empty_like(uk)
    hk.apply(hk.L, uk, out)
    for i in range(K):
        o1 = torch.empty(n, dtype=torch.float64, device="cuda")
        h1.apply(h1.L, to_dev(us[i]), o1)
        assert float((out[i * n:(i + 1) * n] - o1).abs().max() / o1.abs().max()) < 1e-13
    for l in range(1, h1.L + 1):
        nl = h1.ndof(l)
        ul, fl = vectors((nl,), [7, 8, 9]), vectors((nl,), [10, 11, 12])
        ukl = to_dev(np.concatenate(ul))
        hk.smooth(l, ukl, to_dev(np.concatenate(fl)), 1)
        for i in range(K):
            u1 = to_dev(ul[i])
            h1.smooth(l, u1, to_dev(fl[i]), 1)
            assert float((ukl[i * nl:(i + 1) * nl] - u1).abs().max() / u1.abs().max()) < 1e-11, (l, i)
    zk = torch.zeros_like(fk)
    hk.vcycle(fk, zk)
    for i in range(K):
        z1 = torch.zeros(n, dtype=torch.float64, device="cuda")
        h1.vcycle(to_dev(fs[i]), z1)
        assert float((zk[i * n:(i + 1) * n] - z1).abs().max() / z1.abs().max()) < 1e-10


@pytest.mark.parametrize("kind", ["EA", "FA"])
@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_solve_each_rhs_matches_oracle(case, kind):
    dim, P, ne, sp = case
    _, hk = make(case, nrhs=K, smoother=kind)
    oh = OHier(dim, P, sp, False, smoother=kind)
    shape = elem_shape(dim, ne, P)
    Fs = [e2g(f, dim) for f in vectors(shape, [21, 22])] + [np.zeros(oh.fine.shape)]
    refs = [mgcg(oh, np.zeros_like(F), F, rtol=1e-10) for F in Fs[:2]]
    gk = to_dev(np.concatenate([g2e(F, ne, P).reshape(-1) for F in Fs]))
    n = gk.numel() // K
    for run in range(2):                          # host-driven loop, then the device loop
        uk = torch.zeros_like(gk)
        rc, its, hists = hk.solve(gk, uk, rtol=1e-10)
        assert rc == 0 and hk.last_device_loop == (run == 1)
        for i, (U, ohist) in enumerate(refs):
            assert its[i] == len(ohist) - 1, (i, its)
            assert np.allclose(hists[i], ohist, rtol=1e-6, atol=1e-12 * ohist[0])
            assert rel_err(from_dev(uk[i * n:(i + 1) * n], shape), g2e(U, ne, P)) < 1e-10
        assert its[2] == 0 and hk.last_stats[2][0] == 0
        assert float(uk[2 * n:].abs().max()) == 0.0


@pytest.mark.parametrize("kind", ["EA", "FA"])
def test_tf32_multi_rhs(kind):
    from paper_1603_02524_gb300.binding import tc_timeouts
    case = CASES[1]                               # P = 8: 13^3 patches on the tcgen05 kernel
    dim, P, ne, sp = case
    _, hk = make(case, nrhs=K, smoother=kind, precision="mixed_tf32")
    oh = OHier(dim, P, sp, False, smoother=kind)
    shape = elem_shape(dim, ne, P)
    Fs = [e2g(f, dim) for f in vectors(shape, [31, 32, 33])]
    gk = to_dev(np.concatenate([g2e(F, ne, P).reshape(-1) for F in Fs]))
    n = gk.numel() // K
    uk = torch.zeros_like(gk)
    rc, its, _ = hk.solve(gk, uk, rtol=1e-10)
    assert rc == 0
    for i, F in enumerate(Fs):
        U, ohist = mgcg(oh, np.zeros_like(F), F, rtol=1e-10)
        assert its[i] <= len(ohist) - 1 + 2
        assert rel_err(from_dev(uk[i * n:(i + 1) * n], shape), g2e(U, ne, P)) < 1e-9
    assert tc_timeouts() == 0


def test_batch_of_multi_rhs_hierarchies():
    from paper_1603_02524_gb300 import Batch
    hs, gs, us, singles = [], [], [], []
    for j, case in enumerate(CASES[:2]):
        _, hk = make(case, nrhs=2, smoother="FA", variable_v=True)
        _, h1 = make(case, smoother="FA", variable_v=True)
        n = h1.ndof()
        vs = vectors((n,), [40 + 2 * j, 41 + 2 * j])
        hs.append(hk)
        gs.append(to_dev(np.concatenate(vs)))
        us.append(torch.zeros(2 * n, dtype=torch.float64, device="cuda"))
        singles.append((h1, vs))
    b = Batch(hs, gs, us, rtol=1e-10)
    rc, res = b.solve()
    assert rc == 0 and len(res) == 4
    k = 0
    for (h1, vs), u in zip(singles, us):
        n = h1.ndof()
        for i, v in enumerate(vs):
            u1 = torch.zeros(n, dtype=torch.float64, device="cuda")
            rc1, it1, _ = h1.solve(to_dev(v), u1, rtol=1e-10)
            assert rc1 == 0 and res[k][1] == it1 and res[k][0] == 0
            assert float((u[i * n:(i + 1) * n] - u1).abs().max() / u1.abs().max()) < 1e-11
            k += 1
    b.close()


def test_periodic_grid_rejects_several_rhs():
    from paper_1603_02524_gb300 import Grid, Hierarchy, PmgError
    g = Grid(3, 2, (2, 2, 2), [[0.5, 0.5]] * 3, periodic=True)
    with pytest.raises(PmgError):
        Hierarchy(g, nrhs=2)

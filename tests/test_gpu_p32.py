"""GPU parity at P = 32 in 3-D, where an element (33^3 nodes) and a patch (43^3, or
64 x 43 x 43 for the face-centred family) no longer fit shared memory: the operator
apply runs one launch per axis, the transfers between P = 32 and 16 share one
in-place buffer, and the patch solves keep their patch buffer in global scratch.
Tolerances as in test_gpu_parity.py (operator and transfers 1e-13, one Schwarz
step 1e-11, MGCG solution 1e-10 with the oracle's iteration count; fp32 V-cycle
steps 1e-4; double-float apply 1e-12; mixed + double-float solve 1e-9).
"""
import numpy as np
import pytest

import synthetic as syn
from oracle import dg, schwarz
from oracle.mg import Hierarchy as OHier, mgcg
from tests.helpers import e2g, elem_shape, from_dev, g2e, rel_err, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [
    # dim, P, n_elem, spacing, periodic, beta
    (3, 32, (2, 2, 2), [[0.5, 0.5], [0.4, 0.6], [0.5, 0.5]], False, 0.0),
    (3, 32, (2, 2, 2), [[0.5, 0.5], [0.5, 0.5], [0.5, 0.5]], True, 0.5),
]
IDS = ["dir-stretched-ip", "per-uniform-ldg"]


def make(case, **opts):
    from paper_1603_02524_gb300 import Grid, Hierarchy
    dim, P, ne, sp, per, beta = case
    g = Grid(dim, P, ne, sp, periodic=per, beta=beta)
    return g, Hierarchy(g, **opts)


def rnd(shape, seed):
    return syn.rng(seed).uniform(-1, 1, size=shape)


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_p32_apply_residual_and_transfers(case):
    dim, P, ne, sp, per, beta = case
    g, h = make(case)
    hdf = make(case, outer_apply="df")[1]
    oh = OHier(dim, P, sp, per, beta)
    for l in range(h.L + 1):
        Pl = 2 ** l
        shape = elem_shape(dim, ne, Pl)
        u, f = rnd(shape, 10 + l), rnd(shape, 20 + l)
        disc = dg.Discretisation(dim, Pl, sp, per, beta, 1.0)
        ref = g2e(disc.apply(e2g(u, dim)), ne, Pl)
        out = torch.empty(int(np.prod(shape)), dtype=torch.float64, device="cuda")
        h.apply(l, to_dev(u), out)
        assert rel_err(from_dev(out, shape), ref) < 1e-13, l
        h.residual(l, to_dev(u), to_dev(f), out)
        assert rel_err(from_dev(out, shape), f - ref) < 1e-13, l
        if l == h.L:
            hdf.apply(l, to_dev(u), out)
            assert rel_err(from_dev(out, shape), ref) < 1e-12
    for l in range(1, h.L + 1):
        sf, sc = elem_shape(dim, ne, 2 ** l), elem_shape(dim, ne, 2 ** (l - 1))
        rf, uc, uf = rnd(sf, 1), rnd(sc, 2), rnd(sf, 3)
        out = torch.empty(int(np.prod(sc)), dtype=torch.float64, device="cuda")
        h.restrict(l, to_dev(rf), out)
        ref = g2e(oh.restrict(l, e2g(rf, dim)), ne, 2 ** (l - 1))
        assert rel_err(from_dev(out, sc), ref) < 1e-13, l
        uft = to_dev(uf)
        h.prolong(l, to_dev(uc), uft)
        ref = uf + g2e(oh.prolong(l, e2g(uc, dim)), ne, 2 ** l)
        assert rel_err(from_dev(uft, sf), ref) < 1e-13, l


@pytest.mark.parametrize("kind,overlap", [("EA", "l"), ("EA", "0"), ("FA", "l"), ("FA", "0")])
@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_p32_smoother_step(case, kind, overlap):
    dim, P, ne, sp, per, beta = case
    g, h = make(case, smoother=kind, overlap=overlap)
    hm = make(case, smoother=kind, overlap=overlap, precision="mixed")[1]
    l = h.L
    shape = elem_shape(dim, ne, P)
    u, f = rnd(shape, 30), rnd(shape, 31)
    disc = dg.Discretisation(dim, P, sp, per, beta, 1.0)
    sm = schwarz.Smoother(disc, kind, overlap, "quintic")
    ref = g2e(sm.step(e2g(u, dim), e2g(f, dim)), ne, P)
    ut = to_dev(u)
    h.smooth(l, ut, to_dev(f), 1)
    assert rel_err(from_dev(ut, shape), ref) < 1e-11
    um = to_dev(u)
    hm.smooth(l, um, to_dev(f), 1)
    assert rel_err(from_dev(um, shape), ref) < 1e-4


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_p32_mgcg(case):
    dim, P, ne, sp, per, beta = case
    g, h = make(case)
    shape = elem_shape(dim, ne, P)
    F = e2g(rnd(shape, 40), dim)
    if per:
        F -= F.mean()
    oh = OHier(dim, P, sp, per, beta)
    U, ohist = mgcg(oh, np.zeros_like(F), F, rtol=1e-10)
    ref = g2e(U, ne, P)
    gt = to_dev(g2e(F, ne, P))
    for run in range(2):                          # host-driven loop, then the device loop
        u = torch.zeros(int(np.prod(shape)), dtype=torch.float64, device="cuda")
        rc, it, hist = h.solve(gt, u, rtol=1e-10)
        assert rc == 0 and it == len(ohist) - 1 and h.last_device_loop == (run == 1)
        got = from_dev(u, shape)
        r = ref
        if per:
            got, r = got - got.mean(), ref - ref.mean()
        assert rel_err(got, r) < 1e-10
    hm = make(case, precision="mixed", outer_apply="df")[1]
    hm.autotune()
    u = torch.zeros(int(np.prod(shape)), dtype=torch.float64, device="cuda")
    rc, it, hist = hm.solve(gt, u, rtol=1e-10)
    assert rc == 0 and abs(it - (len(ohist) - 1)) <= 1
    got = from_dev(u, shape)
    if per:
        got = got - got.mean()
        ref = ref - ref.mean()
    assert rel_err(got, ref) < 1e-9


@pytest.mark.parametrize("kind", ["EA", "FA"])
def test_p32_mgcg_autotuned(kind):
    """The tuner times both forms of the large-patch kernel per family (scratch buffer, or
    slabs of c-planes in shared memory) and keeps the faster: FP64 solves with its choice
    against the oracle (iteration count, solution to 1e-10)."""
    case = CASES[0]
    dim, P, ne, sp, per, beta = case
    g, h = make(case, smoother=kind)
    h.autotune()
    shape = elem_shape(dim, ne, P)
    F = e2g(rnd(shape, 41), dim)
    oh = OHier(dim, P, sp, per, beta, smoother=kind)
    U, ohist = mgcg(oh, np.zeros_like(F), F, rtol=1e-10)
    u = torch.zeros(int(np.prod(shape)), dtype=torch.float64, device="cuda")
    rc, it, _ = h.solve(to_dev(g2e(F, ne, P)), u, rtol=1e-10)
    assert rc == 0 and it == len(ohist) - 1
    assert rel_err(from_dev(u, shape), g2e(U, ne, P)) < 1e-10

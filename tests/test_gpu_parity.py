"""GPU parity: every step of the CUDA path against the FP64 CPU oracle, element by element.

FP64 mode tolerances (relative to the max-norm of the oracle result):
  operator apply / mass / transfers      1e-13  (a few dozen rounded FMAs per entry)
  one Schwarz step                       1e-11  (eigen-tables from two different
                                                 eigen-solvers; kappa(L_s) ~ 1e4-1e6)
  coarse solve, V-cycle                  1e-10
  full MGCG solve (rtol 1e-10)           1e-10 of the solution, equal iteration counts
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
    (2, 4, (4, 4), [[0.25] * 4, [0.25] * 4], False, 0.0),
    (2, 8, (3, 4), [[0.3, 0.5, 0.2], [0.4, 0.1, 0.3, 0.2]], True, 0.5),
    (2, 16, (3, 2), [[0.3, 0.5, 0.2], [0.6, 0.4]], False, 0.0),
    (3, 2, (3, 2, 4), [[0.3, 0.5, 0.2], [0.6, 0.4], [0.1, 0.2, 0.3, 0.4]], False, 0.5),
    (3, 4, (3, 3, 2), [[0.3, 0.5, 0.2], [0.2, 0.3, 0.5], [0.6, 0.4]], True, 0.0),
    (3, 8, (2, 3, 2), [[0.5, 0.5], [0.3, 0.3, 0.4], [0.7, 0.3]], False, 0.0),
    (3, 16, (2, 1, 2), [[0.5, 0.5], [1.0], [0.5, 0.5]], False, 0.5),
    # uniform grids: interior patches are centro-symmetric (even-odd split in the kernel)
    (3, 8, (4, 3, 3), [[0.25] * 4, [1 / 3] * 3, [1 / 3] * 3], False, 0.0),
    (3, 4, (3, 4, 3), [[1 / 3] * 3, [0.25] * 4, [1 / 3] * 3], True, 0.0),
    (2, 8, (5, 4), [[0.2] * 5, [0.25] * 4], True, 0.0),
]
IDS = [f"{c[0]}d-P{c[1]}-{'x'.join(map(str, c[2]))}-{'per' if c[4] else 'dir'}-b{c[5]}" for c in CASES]


def make(case, **opts):
    from paper_1603_02524_gb300 import Grid, Hierarchy
    dim, P, ne, sp, per, beta = case
    g = Grid(dim, P, ne, sp, periodic=per, beta=beta)
    h = Hierarchy(g, **opts)
    return g, h


def rnd(shape, seed):
    return syn.rng(seed).uniform(-1, 1, size=shape)


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_apply_and_residual(case):
    dim, P, ne, sp, per, beta = case
    g, h = make(case)
    for l in range(h.L + 1):
        Pl = 2 ** l
        shape = elem_shape(dim, ne, Pl)
        u = rnd(shape, 10 + l)
        f = rnd(shape, 20 + l)
        disc = dg.Discretisation(dim, Pl, sp, per, beta, 1.0)
        ref = g2e(disc.apply(e2g(u, dim)), ne, Pl)
        ut, ft = to_dev(u), to_dev(f)
        out = torch.empty_like(ut)
        h.apply(l, ut, out)
        assert rel_err(from_dev(out, shape), ref) < 1e-13
        h.residual(l, ut, ft, out)
        assert rel_err(from_dev(out, shape), f - ref) < 1e-13


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_rhs_mass(case):
    dim, P, ne, sp, per, beta = case
    g, h = make(case)
    shape = elem_shape(dim, ne, P)
    f = rnd(shape, 3)
    disc = dg.Discretisation(dim, P, sp, per, beta, 1.0)
    ref = g2e(disc.rhs(e2g(f, dim)), ne, P)
    out = torch.empty(int(np.prod(shape)), dtype=torch.float64, device="cuda")
    h.rhs(to_dev(f), out)
    assert rel_err(from_dev(out, shape), ref) < 1e-14


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_transfers(case):
    dim, P, ne, sp, per, beta = case
    g, h = make(case)
    oh = OHier(dim, P, sp, per, beta)
    for l in range(1, h.L + 1):
        sf, sc = elem_shape(dim, ne, 2 ** l), elem_shape(dim, ne, 2 ** (l - 1))
        rf, uc, uf = rnd(sf, 1), rnd(sc, 2), rnd(sf, 3)
        out = torch.empty(int(np.prod(sc)), dtype=torch.float64, device="cuda")
        h.restrict(l, to_dev(rf), out)
        ref = g2e(oh.restrict(l, e2g(rf, dim)), ne, 2 ** (l - 1))
        assert rel_err(from_dev(out, sc), ref) < 1e-13
        uft = to_dev(uf)
        h.prolong(l, to_dev(uc), uft)
        ref = uf + g2e(oh.prolong(l, e2g(uc, dim)), ne, 2 ** l)
        assert rel_err(from_dev(uft, sf), ref) < 1e-13


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_coarse_solve(case):
    dim, P, ne, sp, per, beta = case
    g, h = make(case)
    oh = OHier(dim, P, sp, per, beta, coarse="dense")
    shape = elem_shape(dim, ne, 1)
    f0 = rnd(shape, 4)
    if per:
        f0 -= f0.mean()
    out = torch.empty(int(np.prod(shape)), dtype=torch.float64, device="cuda")
    h.coarse_solve(to_dev(f0), out)
    got = from_dev(out, shape)
    ref = g2e(oh.coarse_solve(e2g(f0, dim)), ne, 1)
    if per:                      # solutions differ by a null-space constant
        got, ref = got - got.mean(), ref - ref.mean()
    assert rel_err(got, ref) < 1e-10


SMOOTH = [("EA", "l"), ("EA", "0"), ("FA", "l"), ("FA", "0")]


@pytest.mark.parametrize("kind,overlap", SMOOTH)
@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_smoother_step(case, kind, overlap):
    dim, P, ne, sp, per, beta = case
    if P == 16 and dim == 3 and kind == "FA" and overlap == "0":
        pass
    g, h = make(case, smoother=kind, overlap=overlap, weighting="quintic")
    for l in range(1, h.L + 1):
        Pl = 2 ** l
        shape = elem_shape(dim, ne, Pl)
        u, f = rnd(shape, 5 + l), rnd(shape, 6 + l)
        disc = dg.Discretisation(dim, Pl, sp, per, beta, 1.0)
        sm = schwarz.Smoother(disc, kind, overlap, "quintic")
        ref = g2e(sm.step(e2g(u, dim), e2g(f, dim)), ne, Pl)
        ut = to_dev(u)
        h.smooth(l, ut, to_dev(f), 1)
        assert rel_err(from_dev(ut, shape), ref) < 1e-11, (l, kind, overlap)


@pytest.mark.parametrize("weighting", ["unweighted", "arithmetic", "cubic"])
def test_smoother_weightings(weighting):
    case = CASES[4]
    dim, P, ne, sp, per, beta = case
    for kind in ("EA", "FA"):
        g, h = make(case, smoother=kind, overlap="l", weighting=weighting)
        shape = elem_shape(dim, ne, P)
        u, f = rnd(shape, 7), rnd(shape, 8)
        disc = dg.Discretisation(dim, P, sp, per, beta, 1.0)
        sm = schwarz.Smoother(disc, kind, "l", weighting)
        ref = g2e(sm.step(e2g(u, dim), e2g(f, dim)), ne, P)
        ut = to_dev(u)
        h.smooth(h.L, ut, to_dev(f), 1)
        assert rel_err(from_dev(ut, shape), ref) < 1e-11


@pytest.mark.parametrize("kind", ["EA", "FA"])
@pytest.mark.parametrize("case", CASES[:6], ids=IDS[:6])
def test_vcycle(case, kind):
    dim, P, ne, sp, per, beta = case
    g, h = make(case, smoother=kind)
    oh = OHier(dim, P, sp, per, beta, smoother=kind, coarse="dense")
    shape = elem_shape(dim, ne, P)
    f = rnd(shape, 9)
    F = e2g(f, dim)
    if per:
        F -= F.mean()
        f = g2e(F, ne, P)
    out = torch.zeros(int(np.prod(shape)), dtype=torch.float64, device="cuda")
    h.vcycle(to_dev(f), out)
    got = from_dev(out, shape)
    ref = g2e(oh.vcycle(np.zeros_like(F), F), ne, P)
    if per:
        got, ref = got - got.mean(), ref - ref.mean()
    assert rel_err(got, ref) < 1e-10


@pytest.mark.parametrize("kind", ["EA", "FA"])
@pytest.mark.parametrize("case", CASES[:6], ids=IDS[:6])
def test_mgcg_solve(case, kind):
    dim, P, ne, sp, per, beta = case
    g, h = make(case, smoother=kind)
    oh = OHier(dim, P, sp, per, beta, smoother=kind)
    shape = elem_shape(dim, ne, P)
    f = rnd(shape, 11)
    F = e2g(f, dim)
    if per:
        F -= F.mean()
    U, ohist = mgcg(oh, np.zeros_like(F), F, rtol=1e-10)
    ref = g2e(U, ne, P)
    u = torch.zeros(int(np.prod(shape)), dtype=torch.float64, device="cuda")
    rc, iters, hist = h.solve(to_dev(g2e(F, ne, P)), u, rtol=1e-10)
    assert rc == 0
    assert iters == len(ohist) - 1
    assert np.allclose(hist, ohist, rtol=1e-6, atol=1e-12 * ohist[0])
    got = from_dev(u, shape)
    if per:
        got, ref = got - got.mean(), ref - ref.mean()
    assert rel_err(got, ref) < 1e-10


@pytest.mark.parametrize("outer", ["fp64", "df"])
@pytest.mark.parametrize("case", [CASES[0], CASES[3]], ids=[IDS[0], IDS[3]])
def test_mgcg_solve_from_nonzero_initial_guess(case, outer):
    """Algorithm 2 from a seeded nonzero u_0: the initial residual g - A u_0 is formed by the
    operator apply (a zero u_0 takes the shortcut r_0 = g), in the host-driven loop and in
    the device-side loop, against the oracle's solve from the same u_0."""
    dim, P, ne, sp, per, beta = case
    g, h = make(case, smoother="EA", outer_apply=outer)
    oh = OHier(dim, P, sp, per, beta, smoother="EA")
    shape = elem_shape(dim, ne, P)
    F = e2g(rnd(shape, 13), dim)
    U0 = e2g(rnd(shape, 14), dim)
    if per:
        F -= F.mean()
    U, ohist = mgcg(oh, U0.copy(), F, rtol=1e-10)
    ref = g2e(U, ne, P)
    for run in range(2):                          # host-driven loop, then the device loop
        u = to_dev(g2e(U0, ne, P))
        rc, iters, hist = h.solve(to_dev(g2e(F, ne, P)), u, rtol=1e-10)
        assert rc == 0 and h.last_device_loop == (run == 1)
        assert iters == len(ohist) - 1
        assert np.allclose(hist, ohist, rtol=1e-6, atol=1e-12 * ohist[0])
        got = from_dev(u, shape)
        if per:
            got, ref2 = got - got.mean(), ref - ref.mean()
        else:
            ref2 = ref
        assert rel_err(got, ref2) < 1e-10


def test_config1_manufactured_solution():
    """2-D unit square, 4x4 elements, P=4, IP, Dirichlet, f = 2 pi^2 sin sin: solve, compare."""
    from paper_1603_02524_gb300 import Grid, Hierarchy
    w = syn.config1()
    g = Grid(2, w.P, w.n_elem, w.spacing, periodic=False)
    h = Hierarchy(g, smoother="EA", overlap="l")
    f = syn.source_values(w, [g.coords(0), g.coords(1)])
    ft = to_dev(f)
    gt = torch.empty_like(ft)
    h.rhs(ft, gt)
    u = torch.zeros_like(gt)
    rc, iters, hist = h.solve(gt, u, rtol=1e-10)
    assert rc == 0 and hist[-1] <= 1e-10 * hist[0]
    oh = OHier(2, w.P, w.spacing, False)
    d = oh.fine
    F = d.rhs(d.nodal(syn.sin_source(2)))
    U, ohist = mgcg(oh, np.zeros_like(F), F, rtol=1e-10)
    assert iters == len(ohist) - 1
    got = from_dev(u, elem_shape(2, w.n_elem, w.P))
    assert rel_err(got, g2e(U, w.n_elem, w.P)) < 1e-10
    exact = g2e(d.nodal(syn.sin_solution(2)), w.n_elem, w.P)
    assert np.abs(got - exact).max() < 2e-3          # discretisation error at P = 4, h = 1/4


def test_invalid_arguments():
    from paper_1603_02524_gb300 import PmgError
    case = CASES[0]
    g, h = make(case)
    u = torch.zeros(10, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        h.apply(0, u, u)
    from paper_1603_02524_gb300 import binding
    lib = binding.load()
    assert lib.pmg_apply(h.handle, 99, None, None, None) == -1
    assert lib.pmg_smooth(h.handle, 0, None, None, 1, None) == -1


@pytest.mark.parametrize("kind", ["EA", "FA"])
def test_per_level_parameters(kind):
    """Per-level damping omega_l and transition width tau_l (learned-parameter knobs):
    smoothing steps and a full V-cycle against the oracle with the same parameters."""
    case = CASES[7]                       # uniform 3-D, P = 8: even-odd path with narrowed weights
    dim, P, ne, sp, per, beta = case
    omega_level = [0.0, 0.85, 1.1, 0.9]
    tau_level = [0.0, 0.5, 0.75, 0.3]
    g, h = make(case, smoother=kind, omega_level=omega_level, tau_level=tau_level)
    for l in range(1, h.L + 1):
        shape = elem_shape(dim, ne, 2 ** l)
        u, f = rnd(shape, 30 + l), rnd(shape, 40 + l)
        disc = dg.Discretisation(dim, 2 ** l, sp, per, beta, 1.0)
        sm = schwarz.Smoother(disc, kind, "l", "quintic", omega=omega_level[l], tau=tau_level[l])
        ref = g2e(sm.step(e2g(u, dim), e2g(f, dim)), ne, 2 ** l)
        ut = to_dev(u)
        h.smooth(l, ut, to_dev(f), 1)
        assert rel_err(from_dev(ut, shape), ref) < 1e-11, l
    oh = OHier(dim, P, sp, per, beta, smoother=kind, coarse="dense", omega_level=omega_level,
               tau_level=tau_level)
    shape = elem_shape(dim, ne, P)
    F = e2g(rnd(shape, 50), dim)
    out = torch.zeros(int(np.prod(shape)), dtype=torch.float64, device="cuda")
    h.vcycle(to_dev(g2e(F, ne, P)), out)
    ref = g2e(oh.vcycle(np.zeros_like(F), F), ne, P)
    assert rel_err(from_dev(out, shape), ref) < 1e-10


@pytest.mark.parametrize("precision", ["mixed", "mixed_tc"])
@pytest.mark.parametrize("kind", ["EA", "FA"])
@pytest.mark.parametrize("case", [CASES[5], CASES[6], CASES[7], CASES[8]], ids=[IDS[5], IDS[6], IDS[7], IDS[8]])
def test_mixed_precision_smoother_step(case, kind, precision):
    """fp32 smoothing (SIMT, or tensor cores with the 3xTF32 split) against the FP64 oracle:
    stated per-result error 1e-4 of the correction (fp32 residual and transforms)."""
    dim, P, ne, sp, per, beta = case
    g, h = make(case, smoother=kind, precision=precision)
    for l in range(1, h.L + 1):
        shape = elem_shape(dim, ne, 2 ** l)
        u, f = rnd(shape, 60 + l), rnd(shape, 70 + l)
        disc = dg.Discretisation(dim, 2 ** l, sp, per, beta, 1.0)
        ref = g2e(schwarz.Smoother(disc, kind, "l", "quintic").step(e2g(u, dim), e2g(f, dim)), ne, 2 ** l)
        ut = to_dev(u)
        h.smooth(l, ut, to_dev(f), 1)
        assert rel_err(from_dev(ut, shape) - u, ref - u) < 1e-4, (l, precision)

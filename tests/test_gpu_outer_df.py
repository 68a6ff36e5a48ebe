"""GPU: the CG's operator apply in double-float arithmetic (outer_apply "df").

Each value is carried as the sum of two fp32 words (about 48 significant bits);
products are split exactly with one FMA and sums with TwoSum (Dekker; Knuth;
Ogita-Rump-Oishi's Dot2).  Against the FP64 oracle's operator the apply agrees
to 1e-12 of the result's max-norm: the rounding of the inputs to 48 bits
(2^-48 ~ 3.6e-15) times the cancellation between the stiffness and the face
terms, which reaches a few hundred on stretched elements.  The MGCG solve with
this apply needs the same iterations as the oracle's FP64 solve and reaches the
same solution to 1e-9.
"""
import numpy as np
import pytest

import synthetic as syn
from oracle import dg
from oracle.mg import Hierarchy as OHier, mgcg
from tests.helpers import e2g, elem_shape, from_dev, g2e, rel_err, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [
    (2, 8, (3, 4), [[0.3, 0.5, 0.2], [0.4, 0.1, 0.3, 0.2]], True, 0.5),
    (3, 4, (3, 3, 2), [[0.3, 0.5, 0.2], [0.2, 0.3, 0.5], [0.6, 0.4]], False, 0.0),
    (3, 8, (4, 3, 3), [[0.25] * 4, [1 / 3] * 3, [1 / 3] * 3], False, 0.0),
    (3, 16, (2, 1, 2), [[0.5, 0.5], [1.0], [0.5, 0.5]], False, 0.5),
]
IDS = [f"{c[0]}d-P{c[1]}-{'per' if c[4] else 'dir'}-b{c[5]}" for c in CASES]


def make(case, **opts):
    from paper_1603_02524_gb300 import Grid, Hierarchy
    dim, P, ne, sp, per, beta = case
    g = Grid(dim, P, ne, sp, periodic=per, beta=beta)
    return g, Hierarchy(g, outer_apply="df", **opts)


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_df_apply_and_residual(case):
    dim, P, ne, sp, per, beta = case
    g, h = make(case)
    shape = elem_shape(dim, ne, P)
    disc = dg.Discretisation(dim, P, sp, per, beta, 1.0)
    u = syn.rng(80).uniform(-1, 1, size=shape)
    f = syn.rng(81).uniform(-1, 1, size=shape)
    ref = g2e(disc.apply(e2g(u, dim)), ne, P)
    out = torch.empty(int(np.prod(shape)), dtype=torch.float64, device="cuda")
    h.apply(h.L, to_dev(u), out)
    assert rel_err(from_dev(out, shape), ref) < 1e-12
    h.residual(h.L, to_dev(u), to_dev(f), out)
    assert rel_err(from_dev(out, shape), f - ref) < 1e-12


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_df_mgcg_solve(case):
    dim, P, ne, sp, per, beta = case
    g, h = make(case)
    shape = elem_shape(dim, ne, P)
    F = e2g(syn.rng(82).uniform(-1, 1, size=shape), dim)
    if per:
        F -= F.mean()
    oh = OHier(dim, P, sp, per, beta)
    U, ohist = mgcg(oh, np.zeros_like(F), F, rtol=1e-10)
    gt = to_dev(g2e(F, ne, P))
    for run in range(2):                      # host-driven loop, then the device-side loop
        u = torch.zeros(int(np.prod(shape)), dtype=torch.float64, device="cuda")
        rc, it, hist = h.solve(gt, u, rtol=1e-10)
        assert rc == 0 and h.last_device_loop == (run == 1)
        assert it == len(ohist) - 1
        assert np.allclose(hist, ohist, rtol=1e-6, atol=1e-11 * ohist[0])
        got, ref = from_dev(u, shape), g2e(U, ne, P)
        if per:
            got, ref = got - got.mean(), ref - ref.mean()
        assert rel_err(got, ref) < 1e-9


def test_df_mixed_precision_solve_matches_fp64():
    """Mixed V-cycle with the double-float outer apply vs the all-FP64 solve."""
    from paper_1603_02524_gb300 import Grid, Hierarchy
    w = syn.small_3d(n=(4, 4, 3), P=8)
    g = Grid(3, w.P, w.n_elem, w.spacing, periodic=False)
    h64 = Hierarchy(g)
    hdf = Hierarchy(g, precision="mixed", outer_apply="df")
    shape = elem_shape(3, w.n_elem, w.P)
    gt = to_dev(syn.rng(83).uniform(-1, 1, size=shape))
    u64, udf = torch.zeros_like(gt), torch.zeros_like(gt)
    rc1, it1, _ = h64.solve(gt, u64, rtol=1e-10)
    rc2, it2, hist = hdf.solve(gt, udf, rtol=1e-10)
    assert rc1 == rc2 == 0 and abs(it1 - it2) <= 1
    assert hist[-1] <= 1e-10 * hist[0]
    # the true residual of the double-float solve, in FP64
    r = torch.empty_like(gt)
    h64.residual(h64.L, udf, gt, r)
    assert float(r.norm()) <= 2e-10 * hist[0]
    assert rel_err(from_dev(udf, shape), from_dev(u64, shape)) < 1e-9

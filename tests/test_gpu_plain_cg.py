"""GPU: plain CG (preconditioner "none": z = r in Algorithm 2), the reference method
the paper compares MGCG with in Sec. 4, against the oracle's Algorithm 2 with the
identity as preconditioner.

Hundreds of unpreconditioned iterations amplify rounding differences, so the
iteration counts may differ by a few; the residual histories agree closely in
the first iterations and the solutions agree to 1e-8.
"""
import numpy as np
import pytest

import synthetic as syn
from oracle import dg
from oracle.mg import mgcg
from tests.helpers import e2g, elem_shape, from_dev, g2e, rel_err, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


class IdentityPreconditioner:
    """Stands in for the oracle hierarchy in mgcg: z = r."""

    def __init__(self, disc):
        self.fine = disc

    def vcycle(self, U, R):
        return R.copy()


@pytest.mark.parametrize("dim,P,ne,per", [(2, 4, (4, 3), False), (3, 2, (3, 2, 2), True)])
def test_plain_cg_matches_oracle(dim, P, ne, per):
    from paper_1603_02524_gb300 import Grid, Hierarchy
    sp = [[1.0 / n] * n for n in ne]
    g = Grid(dim, P, ne, sp, periodic=per)
    h = Hierarchy(g, preconditioner="none", max_iter=3000)
    shape = elem_shape(dim, ne, P)
    F = e2g(syn.rng(70).uniform(-1, 1, size=shape), dim)
    if per:
        F -= F.mean()
    disc = dg.Discretisation(dim, P, sp, per, 0.0, 1.0)
    U, ohist = mgcg(IdentityPreconditioner(disc), np.zeros_like(F), F, rtol=1e-10, maxit=3000)
    assert ohist[-1] <= 1e-10 * ohist[0]
    gt = to_dev(g2e(F, ne, P))
    u1 = torch.zeros(int(np.prod(shape)), dtype=torch.float64, device="cuda")
    rc1, it1, h1 = h.solve(gt, u1, rtol=1e-10)
    u2 = torch.zeros_like(u1)
    rc2, it2, h2 = h.solve(gt, u2, rtol=1e-10)                 # device-side loop
    assert rc1 == rc2 == 0 and h.last_device_loop
    assert it1 == it2 and h1 == h2 and torch.equal(u1, u2)     # no atomics without a V-cycle
    assert abs(it1 - (len(ohist) - 1)) <= max(3, (len(ohist) - 1) // 20)
    k = min(10, len(ohist), len(h1))
    assert np.allclose(h1[:k], ohist[:k], rtol=1e-8, atol=0.0)
    got, ref = from_dev(u1, shape), g2e(U, ne, P)
    if per:
        got, ref = got - got.mean(), ref - ref.mean()
    assert rel_err(got, ref) < 1e-8


def test_multigrid_beats_plain_cg():
    """The point of Algorithm 2: far fewer iterations than plain CG on the same problem
    (a random right-hand side, so that CG meets the whole spectrum)."""
    from paper_1603_02524_gb300 import Grid, Hierarchy
    w = syn.config1()
    g = Grid(2, w.P, w.n_elem, w.spacing, periodic=False)
    hm = Hierarchy(g)
    hc = Hierarchy(g, preconditioner="none", max_iter=3000)
    gt = to_dev(syn.rng(71).uniform(-1, 1, size=elem_shape(2, w.n_elem, w.P)))
    um, uc = torch.zeros_like(gt), torch.zeros_like(gt)
    rcm, itm, _ = hm.solve(gt, um, rtol=1e-10)
    rcc, itc, _ = hc.solve(gt, uc, rtol=1e-10)
    assert rcm == rcc == 0
    assert itm * 5 < itc
    assert rel_err(from_dev(uc, (-1,)), from_dev(um, (-1,))) < 1e-8

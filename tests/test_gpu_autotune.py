"""GPU: the patch-kernel autotuner.

The tuner only changes the CTA size of the Schwarz patch kernel; every line
pass strides over its lines by the CTA size, so a tuned sweep must reproduce
the untuned one (to the rounding of the atomic scatter order, 1e-12), and a
tuned hierarchy must still solve to the oracle's solution with the oracle's
iteration count.
"""
import numpy as np
import pytest

import synthetic as syn
from oracle.mg import Hierarchy as OHier, mgcg
from tests.helpers import e2g, elem_shape, from_dev, g2e, rel_err, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CANDIDATES = {64, 96, 128, 160, 192, 256, 320, 384, 448, 512}


@pytest.mark.parametrize("smoother,precision", [("EA", "fp64"), ("FA", "mixed"), ("EA", "mixed_tc")])
def test_autotune_keeps_results(smoother, precision):
    from paper_1603_02524_gb300 import Grid, Hierarchy
    dim, P, ne = 3, 8, (4, 3, 3)
    sp = [[0.25] * 4, [0.2, 0.3, 0.5], [1 / 3] * 3]
    g = Grid(dim, P, ne, sp, periodic=False)
    h = Hierarchy(g, smoother=smoother, precision=precision)
    shape = elem_shape(dim, ne, P)
    fams = [-1] if smoother == "EA" else [0, 1, 2]
    r = to_dev(syn.rng(90).uniform(-1, 1, size=shape))
    before = []
    for fam in fams:
        assert h.tuned_threads(h.L, fam) == 0
        u = torch.zeros_like(r)
        h.schwarz_sweep(h.L, fam, r, u)
        before.append(u)
    F = e2g(syn.rng(91).uniform(-1, 1, size=shape), dim)
    gt = to_dev(g2e(F, ne, P))
    u0 = torch.zeros_like(gt)
    rc0, it0, _ = h.solve(gt, u0, rtol=1e-10)
    u0.zero_()
    h.solve(gt, u0, rtol=1e-10)                 # captured graph, re-captured after tuning
    h.autotune()
    for l in range(1, h.L + 1):
        for fam in fams:
            assert h.tuned_threads(l, fam) in CANDIDATES
    for fam, ub in zip(fams, before):
        u = torch.zeros_like(r)
        h.schwarz_sweep(h.L, fam, r, u)
        tol = 1e-12 if precision == "fp64" else 1e-6
        assert float((u - ub).abs().max()) <= tol * float(ub.abs().max())
    u1 = torch.zeros_like(gt)
    rc1, it1, hist = h.solve(gt, u1, rtol=1e-10)
    assert rc0 == rc1 == 0 and it0 == it1 and h.last_device_loop
    if precision == "fp64":
        oh = OHier(dim, P, sp, False, 0.0, smoother=smoother)
        U, ohist = mgcg(oh, np.zeros_like(F), F, rtol=1e-10)
        assert it1 == len(ohist) - 1
        assert rel_err(from_dev(u1, shape), g2e(U, ne, P)) < 1e-10
    else:
        assert float((u1 - u0).abs().max()) <= 1e-9 * float(u0.abs().max())

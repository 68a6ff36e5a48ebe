"""GPU: the device-detected failure statuses of the solve, each made to happen on purpose
without faulting, trapping or hanging the GPU.

* PMG_ENAN: a NaN placed in the right-hand side on the host makes the initial residual
  non-finite; the host-driven first solve and the device-resident loop (a later solve,
  one CUDA graph) both stop and report it.
* PMG_EBREAKDOWN: a penalty below the coercivity bound (mu_star = -1/2, mu = mu0 / 2)
  leaves the IP operator indefinite (Sec. 2.4 requires mu >= mu0).  Plain CG started
  from u = 0 with g an eigenvector of the most negative eigenvalue (from the oracle's
  dense operator) meets p^T A p < 0 in its first iteration.
* PMG_ETIMEOUT: the tcgen05 patch kernel's bounded waits (PMG_PREC_MIXED_TF32) are made
  to run out by the test hook pmg_test_stall_tc_waits: each block waits on an mbarrier
  that nothing completes, gives up after the stated limit, lets its MMAs finish, frees
  its tensor memory and sets the status.  pmg_solve, pmg_batch_solve and, after
  pmg_smooth, pmg_device_status report it; with the hook off the same hierarchy solves
  normally again.
"""
import numpy as np
import pytest

import synthetic as syn
from oracle import dg
from tests.helpers import e2g, elem_shape, g2e, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PMG_OK, PMG_EBREAKDOWN, PMG_ENAN, PMG_ETIMEOUT = 0, -5, -6, -7


def _grid(P=4, ne=(2, 2, 2), mu_star=1.0):
    from paper_1603_02524_gb300 import Grid
    sp = [[1.0 / n] * n for n in ne]
    return Grid(3, P, ne, sp, periodic=False, mu_star=mu_star), sp


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_nan_in_rhs_gives_enan(precision):
    from paper_1603_02524_gb300 import Hierarchy
    g, _ = _grid()
    h = Hierarchy(g, precision=precision)
    n = h.ndof()
    good = to_dev(syn.rng(1).uniform(-1, 1, n))
    bad = good.clone()
    bad[n // 3] = float("nan")
    u = torch.zeros_like(good)
    rc, it, _ = h.solve(bad, u, check=False)            # first solve: host-driven loop
    assert rc == PMG_ENAN and not h.last_device_loop
    u.zero_()
    rc, _, _ = h.solve(good, u, check=False)
    assert rc == PMG_OK
    u.zero_()
    rc, it, _ = h.solve(bad, u, check=False)            # device-resident loop (one graph)
    assert rc == PMG_ENAN and h.last_device_loop and it == 0
    u.zero_()
    rc, _, _ = h.solve(good, u, check=False)             # the hierarchy stays usable
    assert rc == PMG_OK and h.last_device_loop


def test_indefinite_operator_gives_ebreakdown():
    from paper_1603_02524_gb300 import Hierarchy
    P, ne = 2, (2, 2, 2)
    g, sp = _grid(P, ne, mu_star=-0.5)
    d = dg.Discretisation(3, P, sp, False, 0.0, -0.5)
    lam, vec = np.linalg.eigh(d.dense())
    assert lam[0] < -0.1                               # the operator is indefinite
    G = vec[:, 0].reshape(d.shape)
    gt = to_dev(g2e(G, ne, P))
    h = Hierarchy(g, preconditioner="none")
    for run in range(2):                              # host-driven loop, then the device loop
        u = torch.zeros_like(gt)
        rc, it, _ = h.solve(gt, u, check=False)
        assert rc == PMG_EBREAKDOWN and it == 1 and h.last_device_loop == (run == 1)


def _tc_hier(**opts):
    from paper_1603_02524_gb300 import Hierarchy
    g, _ = _grid(P=8, ne=(2, 2, 2))
    return g, Hierarchy(g, precision="mixed_tf32", **opts)


def test_stalled_tcgen05_wait_gives_etimeout():
    from paper_1603_02524_gb300.binding import tc_timeouts
    g, h = _tc_hier()
    n = h.ndof()
    gt = to_dev(syn.rng(2).uniform(-1, 1, n))
    u = torch.zeros_like(gt)
    rc, it_ok, _ = h.solve(gt, u, check=False)
    assert rc == PMG_OK and tc_timeouts() == 0
    h.test_stall_tc_waits(2000)                        # waits give up after 2 ms
    for run in range(2):                              # the graph was discarded: recaptured, device loop
        u.zero_()
        rc, it, _ = h.solve(gt, u, check=False)
        assert rc == PMG_ETIMEOUT and it == 1 and h.last_device_loop
    assert tc_timeouts() > 0
    # an asynchronous call leaves the status for pmg_device_status
    f = to_dev(syn.rng(3).uniform(-1, 1, n))
    h.smooth(h.L, torch.zeros_like(f), f, 1)
    assert h.device_status() == PMG_ETIMEOUT
    assert h.device_status() == PMG_OK                 # read and reset
    h.test_stall_tc_waits(0)
    assert tc_timeouts() > 0
    u.zero_()
    rc, it, _ = h.solve(gt, u, check=False)
    assert rc == PMG_OK and it == it_ok and tc_timeouts() == 0


def test_stalled_batch_member_reports_etimeout():
    from paper_1603_02524_gb300 import Batch
    from paper_1603_02524_gb300.binding import tc_timeouts
    g, h_bad = _tc_hier()
    _, h_good = _tc_hier()
    n = h_bad.ndof()
    gs = [to_dev(syn.rng(4 + k).uniform(-1, 1, n)) for k in range(2)]
    us = [torch.zeros_like(x) for x in gs]
    h_bad.test_stall_tc_waits(2000)
    b = Batch([h_bad, h_good], gs, us, rtol=1e-10)
    rc, res = b.solve(check=False)
    assert rc == PMG_ETIMEOUT
    assert res[0][0] == PMG_ETIMEOUT and res[1][0] == PMG_OK
    b.close()
    assert tc_timeouts() > 0
    assert tc_timeouts() == 0

"""GPU: the device-resident MGCG loop and batched solves.

Algorithm 2 runs either with host-driven iterations (the first solve of a
hierarchy) or as one CUDA graph whose `while` node repeats the iteration body
and whose condition the convergence test sets on the device (later solves, and
every solve of a batch).  Both issue the same kernels in the same order; the
patch solves scatter their overlapping corrections with atomic adds, whose
order varies from run to run, so iterates agree to rounding (1e-11 relative)
rather than bit for bit, with equal iteration counts.  The device-side loop is
also checked against the FP64 oracle (Algorithm 2 of the paper, same iteration
count, solution within 1e-10).  A batch records several independent solves, of
different grids, orders and right-hand sides, into one graph; each member must
match its own single solve the same way.
"""
import numpy as np
import pytest

import synthetic as syn
from oracle.mg import Hierarchy as OHier, mgcg
from tests.helpers import e2g, elem_shape, from_dev, g2e, rel_err, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def same_run(u_a, u_b, hist_a, hist_b, precision="fp64"):
    """Two runs of one solve: equal iteration counts, iterates equal to rounding.
    FP64 V-cycle: residual histories to 1e-9, solutions to 1e-11.  fp32 V-cycle: the
    atomic order changes the preconditioned residual at fp32 rounding (~1e-7), the
    history by up to ~1e-5 relative, and the converged solutions by far less than
    the 1e-10 stopping tolerance (1e-8 of the solution's max-norm).  tf32 transforms
    (mixed_tf32): the operands are rounded to tf32 between line passes, so an fp32-level
    difference can move a value across a tf32 rounding boundary (2^-11 relative); the
    history may then differ by up to ~1e-2 relative, the solutions as for fp32."""
    assert len(hist_a) == len(hist_b)
    fp64 = precision == "fp64"
    rtol = 1e-9 if fp64 else (2e-2 if precision == "mixed_tf32" else 1e-4)
    assert np.allclose(hist_a, hist_b, rtol=rtol, atol=1e-13 * hist_a[0])
    scale = float(u_a.abs().max()) or 1.0
    assert float((u_a - u_b).abs().max()) <= (1e-11 if fp64 else 1e-8) * scale

CASES = [
    # dim, P, n_elem, spacing, periodic, beta, options
    (3, 4, (3, 2, 4), [[0.3, 0.5, 0.2], [0.6, 0.4], [0.1, 0.2, 0.3, 0.4]], False, 0.0,
     dict(smoother="EA")),
    (3, 8, (3, 3, 2), [[1 / 3] * 3, [0.2, 0.3, 0.5], [0.6, 0.4]], True, 0.5,
     dict(smoother="FA", variable_v=True)),
    (2, 8, (4, 3), [[0.25] * 4, [0.3, 0.3, 0.4]], True, 0.0, dict(smoother="EA", precision="mixed")),
    (3, 8, (4, 3, 3), [[0.25] * 4, [1 / 3] * 3, [1 / 3] * 3], False, 0.0,
     dict(smoother="EA", precision="mixed_tc")),
    # tcgen05 patch kernel (P = 16: 23^3 and 32 x 23 x 23 patches) with the double-float CG apply
    (3, 16, (2, 2, 2), [[0.5, 0.5], [0.4, 0.6], [0.5, 0.5]], True, 0.5,
     dict(smoother="FA", precision="mixed_tf32", outer_apply="df")),
]
IDS = [f"{c[0]}d-P{c[1]}-{'per' if c[4] else 'dir'}-{c[6].get('smoother')}-{c[6].get('precision', 'fp64')}"
       for c in CASES]


def build(case, **extra):
    from paper_1603_02524_gb300 import Grid, Hierarchy
    dim, P, ne, sp, per, beta, opts = case
    g = Grid(dim, P, ne, sp, periodic=per, beta=beta)
    return g, Hierarchy(g, **{**opts, **extra})


def rhs(case, seed):
    dim, P, ne, sp, per, beta, opts = case
    shape = elem_shape(dim, ne, P)
    F = e2g(syn.rng(seed).uniform(-1, 1, size=shape), dim)
    if per:
        F -= F.mean()
    return F, shape


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_device_loop_equals_host_loop_and_oracle(case):
    dim, P, ne, sp, per, beta, opts = case
    g, h = build(case)
    F, shape = rhs(case, 31)
    gt = to_dev(g2e(F, ne, P))
    u1 = torch.zeros(int(np.prod(shape)), dtype=torch.float64, device="cuda")
    rc1, it1, h1 = h.solve(gt, u1, rtol=1e-10)
    assert rc1 == 0 and not h.last_device_loop
    u2 = torch.zeros_like(u1)
    rc2, it2, h2 = h.solve(gt, u2, rtol=1e-10)
    assert rc2 == 0 and h.last_device_loop
    assert it1 == it2
    prec = opts.get("precision", "fp64")
    same_run(u1, u2, h1, h2, prec)
    # replay of the captured graph, and a re-capture for other vectors
    u2.zero_()
    rc, it, hr = h.solve(gt, u2, rtol=1e-10)
    assert (rc, it) == (0, it1)
    same_run(u1, u2, h1, hr, prec)
    u3 = torch.zeros_like(u1)
    rc, it, hr = h.solve(gt, u3, rtol=1e-10)
    assert (rc, it) == (0, it1)
    same_run(u1, u3, h1, hr, prec)
    if opts.get("precision", "fp64") == "fp64":
        oh = OHier(dim, P, sp, per, beta, smoother=opts["smoother"],
                   variable=opts.get("variable_v", False))
        U, ohist = mgcg(oh, np.zeros_like(F), F, rtol=1e-10)
        assert it2 == len(ohist) - 1
        assert np.allclose(h2, ohist, rtol=1e-6, atol=1e-12 * ohist[0])
        got, ref = from_dev(u2, shape), g2e(U, ne, P)
        if per:
            got, ref = got - got.mean(), ref - ref.mean()
        assert rel_err(got, ref) < 1e-10


def test_device_loop_iteration_cap_and_zero_rhs():
    case = CASES[0]
    g, h = build(case, max_iter=2)
    F, shape = rhs(case, 32)
    gt = to_dev(g2e(F, case[2], case[1]))
    u1 = torch.zeros(int(np.prod(shape)), dtype=torch.float64, device="cuda")
    rc1, it1, h1 = h.solve(gt, u1, rtol=1e-14, check=False)
    u2 = torch.zeros_like(u1)
    rc2, it2, h2 = h.solve(gt, u2, rtol=1e-14, check=False)
    assert h.last_device_loop
    assert rc1 == rc2 == -4 and it1 == it2 == 2
    same_run(u1, u2, h1, h2)
    # zero right-hand side and zero guess: r0 = 0, no iteration, u stays 0
    z = torch.zeros_like(gt)
    u3 = torch.zeros_like(u1)
    rc3, it3, h3 = h.solve(z, u3, rtol=1e-10)
    assert (rc3, it3) == (0, 0) and h3 == [0.0]
    assert not torch.any(u3)


def test_batch_equals_single_solves():
    """Grids of different size, order and options; two right-hand sides each."""
    from paper_1603_02524_gb300 import Batch
    members = []
    for ci, case in enumerate(CASES):
        for k in range(2):
            g, h = build(case)
            F, shape = rhs(case, 40 + 2 * ci + k)
            members.append((case, g, h, to_dev(g2e(F, case[2], case[1])), shape))
    # single solves on separate hierarchies of the same configurations
    ref = []
    for case, _, _, gt, shape in members:
        g1, h1 = build(case)
        u = torch.zeros(int(np.prod(shape)), dtype=torch.float64, device="cuda")
        h1.solve(gt, u, rtol=1e-10)
        u.zero_()
        rc, it, hist = h1.solve(gt, u, rtol=1e-10)        # device loop, split coarse solve
        assert rc == 0
        ref.append((u.clone(), it, hist))
    us = [torch.full((int(np.prod(m[4])),), 0.0, dtype=torch.float64, device="cuda") for m in members]
    b = Batch([m[2] for m in members], [m[3] for m in members], us, rtol=1e-10)
    for rep in range(2):
        for u in us:
            u.zero_()
        rc, res = b.solve(history=True)
        assert rc == 0
        for (u_ref, it, hist), u, (st, itb, r0, rn, hb), m in zip(ref, us, res, members):
            assert st == 0 and itb == it
            same_run(u_ref, u, hist, hb, m[0][6].get("precision", "fp64"))
            assert r0 == hb[0] and rn == hb[-1]
            assert r0 == hist[0]
    b.close()


def test_batch_member_matches_oracle():
    from paper_1603_02524_gb300 import Batch
    case = CASES[0]
    dim, P, ne, sp, per, beta, opts = case
    hs, gs, us, Fs = [], [], [], []
    for k in range(3):
        g, h = build(case)
        F, shape = rhs(case, 50 + k)
        hs.append(h)
        gs.append(to_dev(g2e(F, ne, P)))
        us.append(torch.zeros(int(np.prod(shape)), dtype=torch.float64, device="cuda"))
        Fs.append(F)
    b = Batch(hs, gs, us, rtol=1e-10)
    rc, res = b.solve()
    assert rc == 0
    oh = OHier(dim, P, sp, per, beta, smoother="EA")
    for F, u, (st, it, r0, rn) in zip(Fs, us, res):
        U, ohist = mgcg(oh, np.zeros_like(F), F, rtol=1e-10)
        assert it == len(ohist) - 1
        assert abs(r0 - ohist[0]) <= 1e-12 * ohist[0]
        assert rel_err(from_dev(u, elem_shape(dim, ne, P)), g2e(U, ne, P)) < 1e-10


def test_batch_invalid_arguments():
    from paper_1603_02524_gb300 import Batch, PmgError
    case = CASES[0]
    g, h = build(case)
    F, shape = rhs(case, 60)
    gt = to_dev(g2e(F, case[2], case[1]))
    u = torch.zeros_like(gt)
    with pytest.raises(PmgError):
        Batch([h, h], [gt, gt], [u, torch.zeros_like(gt)])    # one workspace, two solves
    with pytest.raises(ValueError):
        Batch([], [], [])
    with pytest.raises(ValueError):
        Batch([h], [gt.float()], [u])

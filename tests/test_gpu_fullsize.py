"""GPU parity at the benchmark sizes.

* 16^3 elements, P = 8 (2 985 984 DOF; the benchmark workload): operator apply,
  one EA step, one FA step and one V-cycle are compared with the oracle on the
  whole vector; the complete MGCG solve is compared on iteration count,
  residual history and solution.
* 32^3 elements, P = 16 (160 989 184 DOF; the mixed-precision workload): the
  oracle cannot hold the problem, so it recomputes sampled outputs one by one on
  local sub-grids around each sampled element (3 x 3 x 3 for A u, 7 x 7 x 7 for one
  EA step), large enough that the sampled outputs are exactly those of the full grid.
Tolerances as in test_gpu_parity.py.
"""
import numpy as np
import pytest

import synthetic as syn
from oracle import dg, schwarz
from oracle.layout import to_element, to_global
from oracle.mg import Hierarchy as OHier, mgcg
from tests.helpers import rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def c2():
    from paper_1603_02524_gb300 import Grid, Hierarchy
    w = syn.config2(0.0)
    g = Grid(3, w.P, w.n_elem, w.spacing, periodic=False)
    f = syn.source_values(w, [g.coords(d) for d in range(3)])
    return w, g, f


def test_c2_apply_ea_step_vcycle(c2):
    from paper_1603_02524_gb300 import Hierarchy
    w, g, f = c2
    h = Hierarchy(g, smoother="EA", overlap="l")
    oh = OHier(3, w.P, w.spacing, False, smoother="EA", overlap="l")
    d = oh.fine
    ne, NP = w.n_elem, w.P + 1
    F = d.rhs(to_global(f, 3))
    ft = torch.from_numpy(to_element(F, ne, NP).reshape(-1)).cuda()
    u = syn.uniform_noise(w, seed=5)
    U = to_global(u, 3)
    ut = torch.from_numpy(u.reshape(-1)).cuda()
    out = torch.empty_like(ut)
    h.apply(h.L, ut, out)
    ref = to_element(d.apply(U), ne, NP)
    assert rel_err(out.cpu().numpy().reshape(ref.shape), ref) < 1e-13
    h.smooth(h.L, ut, ft, 1)
    ref = to_element(oh.levels[oh.L].smoother.step(U, F), ne, NP)
    assert rel_err(ut.cpu().numpy().reshape(ref.shape), ref) < 1e-11
    z = torch.zeros_like(ft)
    h.vcycle(ft, z)
    ref = to_element(oh.vcycle(np.zeros_like(F), F), ne, NP)
    assert rel_err(z.cpu().numpy().reshape(ref.shape), ref) < 1e-10


def test_c2_fa_step(c2):
    from paper_1603_02524_gb300 import Hierarchy
    w, g, f = c2
    h = Hierarchy(g, smoother="FA", overlap="l")
    d = dg.Discretisation(3, w.P, w.spacing, False)
    sm = schwarz.Smoother(d, "FA", "l", "quintic")
    ne, NP = w.n_elem, w.P + 1
    F = d.rhs(to_global(f, 3))
    u = syn.uniform_noise(w, seed=6)
    ut = torch.from_numpy(u.reshape(-1)).cuda()
    h.smooth(h.L, ut, torch.from_numpy(to_element(F, ne, NP).reshape(-1)).cuda(), 1)
    ref = to_element(sm.step(to_global(u, 3), F), ne, NP)
    assert rel_err(ut.cpu().numpy().reshape(ref.shape), ref) < 1e-11


def test_c2_full_solve(c2):
    """The benchmark solve: same iteration count and residual history as the oracle."""
    from paper_1603_02524_gb300 import Hierarchy
    w, g, f = c2
    h = Hierarchy(g, smoother="EA", overlap="l")
    oh = OHier(3, w.P, w.spacing, False, smoother="EA", overlap="l")
    d = oh.fine
    ne, NP = w.n_elem, w.P + 1
    F = d.rhs(to_global(f, 3))
    U, ohist = mgcg(oh, np.zeros_like(F), F, rtol=1e-10)
    ft = torch.from_numpy(f.reshape(-1)).cuda()
    gt = torch.empty_like(ft)
    h.rhs(ft, gt)
    u = torch.zeros_like(gt)
    rc, iters, hist = h.solve(gt, u, rtol=1e-10)
    assert rc == 0 and iters == len(ohist) - 1
    assert np.allclose(hist, ohist, rtol=1e-6, atol=1e-12 * ohist[0])
    ref = to_element(U, ne, NP)
    assert rel_err(u.cpu().numpy().reshape(ref.shape), ref) < 1e-9
    # mixed precision V-cycle: same tolerance reached, solution within 1e-9 of the FP64 oracle
    hm = Hierarchy(g, smoother="EA", overlap="l", precision="mixed")
    um = torch.zeros_like(gt)
    rc, iters_m, hist_m = hm.solve(gt, um, rtol=1e-10)
    assert rc == 0 and hist_m[-1] <= 1e-10 * hist_m[0] and iters_m <= iters + 1
    assert rel_err(um.cpu().numpy().reshape(ref.shape), ref) < 1e-9


# ---------------------------------------------------------------------------
# 32^3 elements, P = 16: sampled outputs on local sub-grids
# ---------------------------------------------------------------------------

def _local_block(u_el, centre, radius, ne):
    """Element-major sub-array of elements centre +- radius (clipped at the walls)."""
    lo = [max(0, c - radius) for c in centre]
    hi = [min(n, c + radius + 1) for c, n in zip(centre, ne)]
    sub = u_el[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]]
    return sub, lo, hi


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_c3_sampled_apply_and_step(precision):
    from paper_1603_02524_gb300 import Grid, Hierarchy
    w = syn.config3()
    ne, P, NP = w.n_elem, w.P, w.P + 1
    h_ = 1.0 / ne[0]
    g = Grid(3, P, ne, w.spacing, periodic=False)
    h = Hierarchy(g, smoother="EA", overlap="l", precision=precision)
    n = h.ndof()
    gen = torch.Generator(device="cuda").manual_seed(7)
    ut = torch.rand(n, dtype=torch.float64, device="cuda", generator=gen) * 2 - 1
    ft = torch.rand(n, dtype=torch.float64, device="cuda", generator=gen) * 2 - 1
    shape = (ne[2], ne[1], ne[0], NP, NP, NP)
    samples = [(0, 0, 0), (31, 0, 17), (15, 16, 14), (3, 30, 31), (20, 9, 1)]
    if precision == "fp64":
        out = torch.empty_like(ut)
        h.apply(h.L, ut, out)
        u_el = ut.view(shape)
        for c in samples:
            sub, lo, hi = _local_block(u_el, c, 1, ne)
            sub = sub.cpu().numpy()
            dims = [hi[k] - lo[k] for k in range(3)]
            d = dg.Discretisation(3, P, [[h_] * dims[k] for k in range(3)], False)
            # the sub-grid walls coincide with the domain walls only where the block was clipped;
            # elsewhere the sampled element is interior to the block and its rows are exact
            if any((lo[k] > 0 and c[k] == lo[k]) or (hi[k] < ne[k] and c[k] == hi[k] - 1) for k in range(3)):
                continue
            ref = to_element(d.apply(to_global(sub, 3)), dims, NP)[c[2] - lo[2], c[1] - lo[1], c[0] - lo[0]]
            got = out.view(shape)[c[2], c[1], c[0]].cpu().numpy()
            assert rel_err(got, ref) < 1e-13
    # one EA step on the whole grid; compare the correction at sampled elements, recomputed
    # by the oracle on a 7 x 7 x 7 element sub-grid: the correction of element c comes from
    # the patches of c and its neighbours, whose residuals need the rows of elements two away,
    # which need the values of elements three away
    u0 = ut.clone()
    h.smooth(h.L, ut, ft, 1)
    # mixed: fp32 residual and transforms; stated per-result error 1e-4 of the correction
    tol = 1e-11 if precision == "fp64" else 1e-4
    u_el, f_el, u1 = u0.view(shape), ft.view(shape), ut.view(shape)
    checked = 0
    for c in samples:
        sub_u, lo, hi = _local_block(u_el, c, 3, ne)
        sub_f, _, _ = _local_block(f_el, c, 3, ne)
        dims = [hi[k] - lo[k] for k in range(3)]
        ok = all((c[k] - lo[k] >= 3 or lo[k] == 0) and (hi[k] - 1 - c[k] >= 3 or hi[k] == ne[k])
                 for k in range(3))
        if not ok:
            continue
        checked += 1
        d = dg.Discretisation(3, P, [[h_] * dims[k] for k in range(3)], False)
        # walls of the sub-grid that are not domain walls would change the patch of the centre
        # element only through elements two away, which the patch does not reach (N_o < P)
        sm = schwarz.Smoother(d, "EA", "l", "quintic")
        Ug = to_global(sub_u.cpu().numpy(), 3)
        Fg = to_global(sub_f.cpu().numpy(), 3)
        new = to_element(sm.step(Ug, Fg), dims, NP)
        ref = new[c[2] - lo[2], c[1] - lo[1], c[0] - lo[0]]
        got = u1[c[2], c[1], c[0]].cpu().numpy()
        base = sub_u.cpu().numpy()[c[2] - lo[2], c[1] - lo[1], c[0] - lo[0]]
        # compare the correction (new - old), relative to its size
        assert rel_err(got - base, ref - base) < tol, (c, precision)
    assert checked >= 4

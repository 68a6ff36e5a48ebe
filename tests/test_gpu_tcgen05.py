"""GPU: the tcgen05 patch kernel (precision "mixed_tf32": the six line passes of each
patch solve as tf32 MMAs, accumulators in tensor memory) against the FP64 oracle.

Tolerance of one smoothing step, relative to the max-norm of the oracle's correction:
the tables are rounded to tf32 (11 significant bits, relative error <= 2^-11 = 4.9e-4),
the gathered residual and the operands between line passes truncated to tf32 (< 2^-10),
and the products summed in fp32; six passes and the scaling compound to a few 2^-10, so
1e-2 bounds the step with margin while any misplaced row,
column or table entry gives errors of order 1.  The fp32 residual of the smoother adds
~1e-7.  The full MGCG solve (FP64 flexible CG, tf32 V-cycle) must reach the oracle's
solution to 1e-9 with at most two more iterations than the oracle.  Every test also
checks that no block of the kernel gave up waiting for its MMAs.
"""
import numpy as np
import pytest

import synthetic as syn
from oracle import dg, schwarz
from oracle.mg import Hierarchy as OHier, mgcg
from tests.helpers import e2g, elem_shape, from_dev, g2e, rel_err, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TF32_STEP_TOL = 1e-2
# patches below 13^3 nodes (P < 8) run the SIMT fp32 kernel in this mode; the P = 2, 4
# levels of these cases therefore check that hand-over as well

CASES = [
    # dim, P, n_elem, spacing, periodic, beta
    (3, 2, (3, 2, 4), [[0.3, 0.5, 0.2], [0.6, 0.4], [0.1, 0.2, 0.3, 0.4]], False, 0.5),
    (3, 4, (3, 3, 2), [[0.3, 0.5, 0.2], [0.2, 0.3, 0.5], [0.6, 0.4]], True, 0.0),
    (3, 8, (2, 3, 2), [[0.5, 0.5], [0.3, 0.3, 0.4], [0.7, 0.3]], False, 0.0),
    (3, 8, (4, 3, 3), [[0.25] * 4, [1 / 3] * 3, [1 / 3] * 3], False, 0.0),
    (3, 16, (2, 2, 2), [[0.5, 0.5], [0.4, 0.6], [0.5, 0.5]], True, 0.5),
]
IDS = [f"P{c[1]}-{'x'.join(map(str, c[2]))}-{'per' if c[4] else 'dir'}-b{c[5]}" for c in CASES]


def make(case, **opts):
    from paper_1603_02524_gb300 import Grid, Hierarchy
    dim, P, ne, sp, per, beta = case
    return Hierarchy(Grid(dim, P, ne, sp, periodic=per, beta=beta), **opts)


def rnd(shape, seed):
    return syn.rng(seed).uniform(-1, 1, size=shape)


def no_timeouts():
    from paper_1603_02524_gb300.binding import tc_timeouts
    return tc_timeouts() == 0


@pytest.mark.parametrize("kind", ["EA", "FA"])
@pytest.mark.parametrize("case,overlap", [(c, "l") for c in CASES] + [(CASES[4], "0")],
                         ids=IDS + [IDS[4] + "-overlap0"])
def test_tf32_smoother_step(case, overlap, kind):
    """Overlap 0 at P = 16 gives the 17^3 and 32 x 17 x 17 patch shapes."""
    dim, P, ne, sp, per, beta = case
    h = make(case, smoother=kind, precision="mixed_tf32", overlap=overlap)
    hs = make(case, smoother=kind, precision="mixed", overlap=overlap)
    for l in range(1, h.L + 1):
        shape = elem_shape(dim, ne, 2 ** l)
        u, f = rnd(shape, 60 + l), rnd(shape, 70 + l)
        disc = dg.Discretisation(dim, 2 ** l, sp, per, beta, 1.0)
        ref = g2e(schwarz.Smoother(disc, kind, overlap, "quintic").step(e2g(u, dim), e2g(f, dim)), ne, 2 ** l)
        ut = to_dev(u)
        h.smooth(l, ut, to_dev(f), 1)
        got = from_dev(ut, shape)
        assert rel_err(got - u, ref - u) < TF32_STEP_TOL, l
        us = to_dev(u)
        hs.smooth(l, us, to_dev(f), 1)                  # SIMT fp32 kernel, same fp32 residual
        assert rel_err(got - u, from_dev(us, shape) - u) < TF32_STEP_TOL, l
    assert no_timeouts()


@pytest.mark.parametrize("kind", ["EA", "FA"])
def test_tf32_sweep_is_linear_and_local(kind):
    """One sweep on a unit residual at a single node changes u only inside the patches
    that contain the node, and scales linearly (a zero residual gives a zero sweep)."""
    case = CASES[3]
    dim, P, ne, sp, per, beta = case
    h = make(case, smoother=kind, precision="mixed_tf32")
    shape = elem_shape(dim, ne, P)
    n = int(np.prod(shape))
    fams = [-1] if kind == "EA" else [0, 1, 2]
    for fam in fams:
        r = torch.zeros(n, dtype=torch.float64, device="cuda")
        u = torch.zeros_like(r)
        h.schwarz_sweep(h.L, fam, r, u)
        assert float(u.abs().max()) == 0.0
        r[n // 2 + 7] = 1.0
        h.schwarz_sweep(h.L, fam, r, u)
        u2 = torch.zeros_like(r)
        h.schwarz_sweep(h.L, fam, 2.0 * r, u2)
        assert float(u.abs().max()) > 0.0
        assert float((u2 - 2.0 * u).abs().max()) <= 1e-6 * float(u2.abs().max())
    assert no_timeouts()


@pytest.mark.parametrize("kind", ["EA", "FA"])
@pytest.mark.parametrize("case", [CASES[1], CASES[3], CASES[4]], ids=[IDS[1], IDS[3], IDS[4]])
def test_tf32_mgcg(case, kind):
    dim, P, ne, sp, per, beta = case
    h = make(case, smoother=kind, precision="mixed_tf32")
    shape = elem_shape(dim, ne, P)
    F = e2g(rnd(shape, 40), dim)
    if per:
        F -= F.mean()
    oh = OHier(dim, P, sp, per, beta, smoother=kind)
    U, ohist = mgcg(oh, np.zeros_like(F), F, rtol=1e-10)
    ref = g2e(U, ne, P)
    gt = to_dev(g2e(F, ne, P))
    for run in range(2):                          # host-driven loop, then the device loop
        u = torch.zeros(int(np.prod(shape)), dtype=torch.float64, device="cuda")
        rc, it, hist = h.solve(gt, u, rtol=1e-10)
        assert rc == 0 and it <= len(ohist) - 1 + 2 and h.last_device_loop == (run == 1)
        got, r = from_dev(u, shape), ref
        if per:
            got, r = got - got.mean(), ref - ref.mean()
        assert rel_err(got, r) < 1e-9
    assert no_timeouts()


def test_tf32_autotune_keeps_results():
    case = CASES[3]
    dim, P, ne, sp, per, beta = case
    h = make(case, smoother="EA", precision="mixed_tf32")
    shape = elem_shape(dim, ne, P)
    r = to_dev(rnd(shape, 90))
    u0 = torch.zeros_like(r)
    h.schwarz_sweep(h.L, -1, r, u0)
    h.autotune()
    for l in range(1, h.L + 1):
        # patches of 13^3 nodes and more run the tcgen05 kernel (CTA 128 ... 512 threads),
        # smaller ones the SIMT kernel
        tc = (2 ** l + 1 + 2 * (1 + round(2 ** l / 8))) >= 13
        assert h.tuned_threads(l, -1) in ((128, 256, 384, 512) if tc else (64, 96, 128, 160, 192, 256, 320, 384, 448, 512))
    u1 = torch.zeros_like(r)
    h.schwarz_sweep(h.L, -1, r, u1)
    assert float((u1 - u0).abs().max()) <= 1e-6 * float(u0.abs().max())
    assert no_timeouts()


@pytest.mark.parametrize("kind", ["EA", "FA"])
@pytest.mark.parametrize("P,ne,per", [(8, 12, False), (16, 8, True)], ids=["P8-12cube-dir", "P16-8cube-per"])
def test_tf32_chunked_patches_match_simt(P, ne, per, kind):
    """Grids with more patches than resident CTAs: each CTA walks a chunk of consecutive
    patches and keeps the tables, eigenvalues and offsets of unchanged axis positions.
    Element widths vary along every axis, so positions differ in their tables.  One
    smoothing step against the SIMT fp32 kernel (itself checked against the oracle)."""
    rng = syn.rng(5 + P)
    sp = []
    for _ in range(3):
        w = rng.uniform(0.5, 2.0, size=ne)
        sp.append(list(w / w.sum()))
    case = (3, P, (ne,) * 3, sp, per, 0.0)
    h = make(case, smoother=kind, precision="mixed_tf32")
    hs = make(case, smoother=kind, precision="mixed")
    shape = elem_shape(3, (ne,) * 3, P)
    u, f = rnd(shape, 80), rnd(shape, 81)
    if per:
        f -= f.mean()
    ut, us = to_dev(u), to_dev(u)
    h.smooth(h.L, ut, to_dev(f), 1)
    hs.smooth(hs.L, us, to_dev(f), 1)
    du, ds = from_dev(ut, shape) - u, from_dev(us, shape) - u
    assert rel_err(du, ds) < TF32_STEP_TOL
    assert no_timeouts()

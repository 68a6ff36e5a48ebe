"""Pins of the oracle's multigrid (Sec. 3.2-3.3) against exact solves and the paper's tables."""
import os

import numpy as np
import pytest

import synthetic as syn
from oracle import dg
from oracle.mg import Hierarchy, cg, interpolation_1d, mg, mgcg, rates

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_tables.txt")


def test_interpolation_reproduces_coarse_polynomials():
    for Pc, Pf in [(1, 2), (2, 4), (4, 8), (8, 16), (16, 32)]:
        J = interpolation_1d(Pc, Pf)
        ec, _ = dg.gll(Pc)
        ef, _ = dg.gll(Pf)
        for k in range(Pc + 1):
            assert np.abs(J @ ec ** k - ef ** k).max() < 1e-11
        assert np.abs(J.sum(axis=1) - 1).max() < 1e-12


def test_restriction_is_transpose_of_prolongation():
    h = Hierarchy(2, 4, [[0.5] * 3, [0.3, 0.7]], False)
    rng = np.random.default_rng(0)
    uc = rng.standard_normal(h.levels[1].disc.shape)
    rf = rng.standard_normal(h.levels[2].disc.shape)
    assert abs(np.vdot(h.prolong(2, uc), rf) - np.vdot(uc, h.restrict(2, rf))) < 1e-12


@pytest.mark.parametrize("periodic", [True, False])
def test_coarse_cg_matches_pseudoinverse(periodic):
    h = Hierarchy(2, 2, [[0.5] * 4, [0.3, 0.3, 0.4]], periodic, coarse="cg")
    d0 = h.levels[0].disc
    rng = np.random.default_rng(1)
    F0 = rng.standard_normal(d0.shape)
    got = h.coarse_solve(F0)
    Fp = F0 - F0.mean() if periodic else F0
    ref = (np.linalg.pinv(d0.dense(), rcond=1e-10, hermitian=True) @ Fp.reshape(-1)).reshape(F0.shape)
    assert np.abs(got - ref).max() < 1e-11 * np.abs(ref).max()


@pytest.mark.parametrize("smoother", ["EA", "FA"])
@pytest.mark.parametrize("periodic", [False, True])
@pytest.mark.parametrize("dim", [2, 3])
def test_mgcg_converges_to_exact_discrete_solution(smoother, periodic, dim):
    sp = [[0.3, 0.4, 0.3], [0.5, 0.25, 0.25], [0.5, 0.5]][:dim]
    P = 4 if dim == 2 else 2
    h = Hierarchy(dim, P, sp, periodic, beta=0.5 if dim == 3 else 0.0, smoother=smoother)
    d = h.fine
    rng = np.random.default_rng(2)
    F = rng.standard_normal(d.shape)
    if periodic:
        F -= F.mean()
    U, hist = mgcg(h, np.zeros_like(F), F, rtol=1e-12, maxit=50)
    assert hist[-1] <= 1e-12 * hist[0]
    ref = np.linalg.lstsq(d.dense(), F.reshape(-1), rcond=1e-10)[0]
    if periodic:
        ref -= ref.mean()
        U = U - U.mean()
    assert np.abs(U.reshape(-1) - ref).max() < 1e-9 * np.abs(ref).max()


def _golden_rows():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        src, meth, sm, P, n, beta, ar, cyc, rbar, n10 = line.split()
        rows.append((src, meth, sm, int(P), int(n), float(beta), int(ar), cyc, float(rbar),
                     None if n10 == "-" else int(n10)))
    return rows


def _paper_hierarchy(sm, P, n, beta=0.0, aspect=1, variable=False):
    kind, ov = sm[:2], sm[2:]
    w = syn.paper_periodic_2d(n, P, aspect=aspect, beta=beta)
    h = Hierarchy(2, P, w.spacing, True, beta=beta, smoother=kind, overlap=ov, weighting="quintic",
                  variable=variable)
    return w, h


def _paper_run(meth, w, h):
    from oracle.layout import to_global
    d = h.fine
    F = d.rhs(d.nodal(syn.sin_source(2)))
    F -= F.mean()
    U0 = to_global(syn.unit_uniform(w, seed=1), 2)
    U, hist = (mgcg if meth == "MGCG" else mg)(h, U0, F, rtol=1e-10, maxit=150)
    return rates(hist)


def _row_id(r):
    src, meth, sm, P, n, beta, ar, cyc = r[:8]
    return f"{src}-{meth}-{sm}-P{P}-n{n}" + (f"-b{beta}" if beta else "") + (f"-AR{ar}" if ar != 1 else "") \
        + ("-varV" if cyc == "VV" else "")


@pytest.mark.parametrize("row", _golden_rows(), ids=_row_id)
def test_paper_convergence_rates(row):
    """Tables 2, 3 and 4 (Sec. 4.3): n10 within +-1 and rbar within 15 %.  Table 3 shows the
    rates are h-independent; its 8 x 8 rows run as printed, Tables 2 and 4 on 16 x 16."""
    src, meth, sm, P, n, beta, ar, cyc, rbar, n10 = row
    w, h = _paper_hierarchy(sm, P, n, beta, ar, variable=(cyc == "VV"))
    got = _paper_run(meth, w, h)
    assert abs(got["rbar"] - rbar) <= 0.15 * rbar, got
    if n10 is not None:
        assert got["n10"] is not None and abs(got["n10"] - n10) <= 1, got


@pytest.mark.parametrize("mistake", ["reversed", "fixed"])
def test_variable_vcycle_pin_catches_a_wrong_schedule(mistake):
    """Plants a plausible mistake in the oracle's variable V-cycle (Table 4, FA_0, P = 4,
    AR = 16, printed n10 = 34): the smoothing steps doubled towards the FINE levels,
    n_{s,l} = 2^(l-1), or not doubled at all.  The Table 4 pin (n10 within +-1) must reject
    both, while the correct schedule n_{s,l} = 2^(L-l) passes."""
    w, h = _paper_hierarchy("FA0", 4, 16, aspect=16, variable=True)
    assert [lev.ns for lev in h.levels] == [(0, 0), (2, 2), (1, 1)]
    if mistake == "reversed":
        good = _paper_run("MGCG", w, h)
        assert abs(good["n10"] - 34) <= 1
    for l, lev in enumerate(h.levels):
        if l > 0:
            k = 2 ** (l - 1) if mistake == "reversed" else 1
            lev.ns = (k, k)
    bad = _paper_run("MGCG", w, h)
    assert abs(bad["n10"] - 34) > 1, bad


def test_printed_overlap_formula_misses_table3_at_P4():
    """Reading C19: with N_o = 1 + floor(P_l/8) (as printed) EA_l at P = 4 needs 8 cycles,
    where Table 3 prints 6; the rounded formula (default 'l') gives 6."""
    w = syn.paper_periodic_2d(8, 4)
    out = {}
    for ov in ("lf", "l"):
        h = Hierarchy(2, 4, w.spacing, True, smoother="EA", overlap=ov)
        d = h.fine
        F = d.rhs(d.nodal(syn.sin_source(2)))
        F -= F.mean()
        from oracle.layout import to_global
        U, hist = mgcg(h, to_global(syn.unit_uniform(w, seed=1), 2), F, rtol=1e-10)
        out[ov] = rates(hist)["n10"]
    assert out["l"] == 6 and out["lf"] >= 8


def test_rates_metric():
    hist = [1.0, 1e-2, 1e-4, 1e-6, 1e-8, 1e-10, 1e-11]
    r = rates(hist)
    assert r["n10"] == 5 and abs(r["rbar"] - 2.0) < 1e-12

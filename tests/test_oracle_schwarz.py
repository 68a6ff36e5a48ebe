"""Pins of the oracle's Schwarz smoothers (Sec. 3.1): weights, FDM local solves."""
import numpy as np
import pytest

from oracle import dg, schwarz


@pytest.mark.parametrize("kind,deg", [("cubic", 3), ("quintic", 5)])
def test_transition_function_conditions(kind, deg):
    # phi~(+-1) = +-1, d^k phi~/dx^k (+-1) = 0 for 0 < k <= (deg-1)/2, strictly monotone (Sec. 3.1)
    x = np.linspace(-1, 1, 2001)
    p = schwarz.phi(x, kind)
    assert p[0] == -1 and p[-1] == 1
    assert np.all(np.diff(p) > 0)
    # the oracle's phi on [-1, 1] is a polynomial of degree deg: recover it and differentiate
    xs = np.cos(np.pi * (np.arange(deg + 1) + 0.5) / (deg + 1))
    poly = np.polynomial.Polynomial.fit(xs, schwarz.phi(xs, kind), deg, domain=[-1, 1])
    assert np.abs(poly(x) - p).max() < 1e-12
    for k in range(1, (deg - 1) // 2 + 1):
        dk = poly.deriv(k)
        assert abs(dk(1.0)) < 1e-11 and abs(dk(-1.0)) < 1e-11
    assert abs(poly.deriv((deg + 1) // 2)(1.0)) > 1e-3
    assert np.all(schwarz.phi(np.array([1.5, -3.0]), kind) == [1, -1])


def _coverage(disc, sm, normal=None):
    tot = np.zeros(disc.shape)
    for pt in sm.subdomains(normal):
        ix = schwarz._ix(pt)
        np.add.at(tot, ix, schwarz.weight_tensor(pt))
    return tot


@pytest.mark.parametrize("periodic", [True, False])
@pytest.mark.parametrize("weighting", ["arithmetic", "cubic", "quintic"])
@pytest.mark.parametrize("P,overlap", [(2, "l"), (4, "l"), (8, "l"), (8, "0"), (16, "l")])
def test_partition_of_unity(periodic, weighting, P, overlap):
    # sum_s R_s^T w_s R_s 1 = 1 (C5, C6, C18)
    disc = dg.Discretisation(2, P, [[0.25] * 4, [0.5, 0.3, 0.2]], periodic)
    for kind in ("EA", "FA"):
        sm = schwarz.Smoother(disc, kind, overlap, weighting)
        normals = [None] if kind == "EA" else [0, 1]
        for nrm in normals:
            assert np.abs(_coverage(disc, sm, nrm) - 1).max() < 1e-14


@pytest.mark.parametrize("tau", [0.25, 0.5, 0.9])
def test_partition_of_unity_narrowed_transition(tau):
    # the learned-parameter extension narrows the transition zone; weights must still sum to 1
    disc = dg.Discretisation(2, 8, [[0.2, 0.3, 0.5], [0.25] * 4], False)
    for kind in ("EA", "FA"):
        sm = schwarz.Smoother(disc, kind, "l", "quintic", tau=tau)
        for nrm in ([None] if kind == "EA" else [0, 1]):
            assert np.abs(_coverage(disc, sm, nrm) - 1).max() < 1e-14
    # tau = 1 reproduces the paper's weights exactly
    a = schwarz.Smoother(disc, "EA", "l", "quintic")
    b = schwarz.Smoother(disc, "EA", "l", "quintic", tau=1.0)
    assert all(np.array_equal(x.w, y.w) for x, y in zip(a.ec[0], b.ec[0]))


def test_partition_of_unity_single_element_axis():
    # one element between two walls: both transition terms take their wall limit (C18)
    disc = dg.Discretisation(3, 4, [[0.5, 0.5], [1.0], [0.3, 0.3, 0.4]], False)
    for kind in ("EA", "FA"):
        sm = schwarz.Smoother(disc, kind, "l", "quintic")
        for nrm in ([None] if kind == "EA" else [0, 1, 2]):
            assert np.abs(_coverage(disc, sm, nrm) - 1).max() < 1e-14


def test_patch_sizes():
    disc = dg.Discretisation(2, 8, [[0.25] * 4, [0.25] * 4], True)
    sm = schwarz.Smoother(disc, "FA", "l", "quintic")
    assert sm.No == 2
    assert len(sm.ec[0][1].idx) == 9 + 4                 # N_P + 2 N_o
    assert len(sm.fc[0][1].idx) == 2 * 9 - 2             # 2 N_P - 2
    discd = dg.Discretisation(2, 8, [[0.25] * 4, [0.25] * 4], False)
    smd = schwarz.Smoother(discd, "FA", "l", "quintic")
    assert len(smd.ec[0][0].idx) == 9 + 2                # truncated at the wall
    assert len(smd.fc[0][0].idx) == 8                    # C13: wall face, N_P - 1 nodes
    assert len(smd.fc[0]) == 5                           # N_e + 1 faces


@pytest.mark.parametrize("periodic", [True, False])
@pytest.mark.parametrize("dim", [2, 3])
def test_fdm_equals_dense_local_inverse(periodic, dim):
    # A_ss^{-1} r_s by fast diagonalisation equals a dense solve with R_s A R_s^T taken from
    # the assembled global matrix (not from the tensor factors)
    sp = [[0.3, 0.4, 0.3], [0.5, 0.2, 0.3], [0.4, 0.6, 0.5]][:dim]
    P = 4 if dim == 2 else 2
    disc = dg.Discretisation(dim, P, sp, periodic, 0.5, 1.0)
    A = disc.dense()
    glob = np.arange(disc.ndof).reshape(disc.shape)
    rng = np.random.default_rng(3)
    for kind in ("EA", "FA"):
        sm = schwarz.Smoother(disc, kind, "l", "quintic")
        for nrm in ([None] if kind == "EA" else list(range(dim))):
            for pt in sm.subdomains(nrm):
                ids = glob[schwarz._ix(pt)].reshape(-1)
                Ass = A[np.ix_(ids, ids)]
                r = rng.standard_normal(len(ids))
                ref = np.linalg.solve(Ass, r)
                got = schwarz.fdm_solve(pt, r.reshape(glob[schwarz._ix(pt)].shape)).reshape(-1)
                assert np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max()


def test_block_jacobi_when_no_overlap():
    # EA_0 with w = 1 (C6) is block Jacobi: one step equals u + blockdiag(A)^{-1} (f - A u)
    disc = dg.Discretisation(2, 3, [[0.5] * 3, [0.5] * 3], False)
    A = disc.dense()
    NP = 4
    glob = np.arange(disc.ndof).reshape(disc.shape)
    rng = np.random.default_rng(4)
    U = rng.standard_normal(disc.shape)
    F = rng.standard_normal(disc.shape)
    sm = schwarz.Smoother(disc, "EA", "0", "quintic")
    got = sm.step(U, F)
    r = (F - disc.apply(U)).reshape(-1)
    du = np.zeros_like(r)
    for ey in range(3):
        for ex in range(3):
            ids = glob[ey * NP:(ey + 1) * NP, ex * NP:(ex + 1) * NP].reshape(-1)
            du[ids] = np.linalg.solve(A[np.ix_(ids, ids)], r[ids])
    assert np.abs(got.reshape(-1) - (U.reshape(-1) + du)).max() < 1e-12


def test_smoother_reduces_high_frequency_error():
    disc = dg.Discretisation(2, 8, [[0.25] * 4, [0.25] * 4], False)
    rng = np.random.default_rng(5)
    E = rng.standard_normal(disc.shape)
    F = np.zeros(disc.shape)
    for kind in ("EA", "FA"):
        sm = schwarz.Smoother(disc, kind, "l", "quintic")
        E1 = sm.step(E, F)
        # energy norm of the error drops by a large factor for rough errors
        en0 = np.vdot(E, disc.apply(E))
        en1 = np.vdot(E1, disc.apply(E1))
        assert en1 < 0.2 * en0

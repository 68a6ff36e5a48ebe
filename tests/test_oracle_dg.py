"""Pins of the oracle's DG discretisation (Sec. 2) against closed forms and invariants."""
import math

import numpy as np
import pytest

from oracle import dg
from oracle.layout import to_element, to_global


# --- GLL nodes and weights: textbook closed forms and quadrature exactness ----

def test_gll_closed_forms():
    eta, rho = dg.gll(2)
    assert np.allclose(eta, [-1, 0, 1], atol=1e-15)
    assert np.allclose(rho, [1 / 3, 4 / 3, 1 / 3], atol=1e-15)
    eta, rho = dg.gll(3)
    s = 1 / math.sqrt(5)
    assert np.allclose(eta, [-1, -s, s, 1], atol=1e-15)
    assert np.allclose(rho, [1 / 6, 5 / 6, 5 / 6, 1 / 6], atol=1e-15)
    eta, rho = dg.gll(4)
    t = math.sqrt(3 / 7)
    assert np.allclose(eta, [-1, -t, 0, t, 1], atol=1e-15)
    assert np.allclose(rho, [1 / 10, 49 / 90, 32 / 45, 49 / 90, 1 / 10], atol=1e-15)


@pytest.mark.parametrize("P", [1, 2, 3, 4, 7, 8, 16, 32])
def test_gll_quadrature_exact_to_degree_2P_minus_1(P):
    eta, rho = dg.gll(P)
    assert eta[0] == -1.0 and eta[-1] == 1.0
    assert rho[0] == pytest.approx(2.0 / (P * (P + 1)), rel=1e-13)
    for k in range(2 * P):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.dot(rho, eta ** k) - exact) < 1e-13


@pytest.mark.parametrize("P", [1, 2, 4, 8, 16, 32])
def test_diff_matrix(P):
    eta, _ = dg.gll(P)
    D = dg.diff_matrix(eta)
    assert D[0, 0] == pytest.approx(-P * (P + 1) / 4, rel=1e-12)
    assert D[P, P] == pytest.approx(P * (P + 1) / 4, rel=1e-12)
    for k in range(P + 1):      # exact on polynomials of degree <= P
        ref = k * eta ** (k - 1) if k > 0 else np.zeros_like(eta)
        assert np.abs(D @ eta ** k - ref).max() < 1e-10 * max(1, k * k)


def test_std_stiffness_P1():
    eta, rho = dg.gll(1)
    Ls = dg.std_stiffness(rho, dg.diff_matrix(eta))
    assert np.allclose(Ls, [[0.5, -0.5], [-0.5, 0.5]], atol=1e-15)


@pytest.mark.parametrize("P", [2, 4, 8])
def test_std_stiffness_is_exact_integral(P):
    # L^s_ik = int phi_i' phi_k' : check v^T L^s u for u = x^a, v = x^b  -> a b / (a+b-1) * (1 - (-1)^(a+b-1))
    eta, rho = dg.gll(P)
    Ls = dg.std_stiffness(rho, dg.diff_matrix(eta))
    for a in range(1, P + 1):
        for b in range(1, P + 1):
            n = a + b - 1
            exact = a * b * (1 - (-1) ** n) / n
            assert abs(eta ** b @ Ls @ eta ** a - exact) < 1e-10


def test_penalty_closed_form():
    # mu0 = {1/dx} P (P+1) / 2  (Sec. 2.4)
    P = 5
    ax = dg.Axis1D(P, [0.3, 0.7], 0.0, 0.0, True)
    ha, hb = 0.3, 0.7
    mu0 = 0.5 * (1 / ha + 1 / hb) * P * (P + 1) / 2
    assert ax._penalty(0) == pytest.approx(mu0, rel=1e-14)


# --- operator invariants --------------------------------------------------------

SP2 = [[0.3, 0.5, 0.2], [0.4, 0.35, 0.25]]


@pytest.mark.parametrize("periodic", [True, False])
@pytest.mark.parametrize("beta", [0.0, 0.5])
@pytest.mark.parametrize("P", [1, 2, 4])
def test_symmetric_psd_nonuniform(periodic, beta, P):
    d = dg.Discretisation(2, P, SP2, periodic, beta, 1.0)
    A = d.dense()
    assert np.abs(A - A.T).max() <= 1e-13 * np.abs(A).max()     # reading C3 needed on stretched grids
    ev = np.linalg.eigvalsh(0.5 * (A + A.T))
    if periodic:
        assert abs(ev[0]) < 1e-10 * ev[-1] and ev[1] > 1e-6 * ev[-1]
        null = A @ np.ones(A.shape[0])
        assert np.abs(null).max() < 1e-12 * np.abs(A).max()
    else:
        assert ev[0] > 1e-6 * ev[-1]


def test_ip_equals_ldg_at_beta0():
    # the unified flux with beta=0 is IP with mu_IP = mu0 (1 + mu_star) (Sec. 2.4): check the
    # IP flux (Eq. flux:num:sigma:components:IP) explicitly on one face.
    P = 3
    ax = dg.Axis1D(P, [0.5, 0.25, 0.25], 0.0, 1.0, True)
    mu_ip = (1 / (2 * 0.5 * ax.rho[P]) + 1 / (2 * 0.25 * ax.rho[0])) * 2
    assert ax._penalty(0) == pytest.approx(mu_ip, rel=1e-14)
    # LDG, beta = 1/2: bracket = (1+2b)^2/(2 dx_a rho_P) + (1-2b)^2/(2 dx_b rho_0) + mu_LDG,
    # mu_LDG = mu - mu0  (Eq. flux:num:sigma:components:LDG)
    b = 0.5
    ax2 = dg.Axis1D(P, [0.5, 0.25, 0.25], b, 1.0, True)
    mu0 = 1 / (2 * 0.5 * ax2.rho[P]) + 1 / (2 * 0.25 * ax2.rho[0])
    ldg = (1 + 2 * b) ** 2 / (2 * 0.5 * ax2.rho[P]) + (1 - 2 * b) ** 2 / (2 * 0.25 * ax2.rho[0]) + mu0
    assert ax2._penalty(0) == pytest.approx(ldg, rel=1e-14)


@pytest.mark.parametrize("beta", [0.0, 0.5])
@pytest.mark.parametrize("P", [2, 3, 5])
def test_dirichlet_polynomial_reproduction_2d(beta, P):
    # u = x(1-x) y(1-y) lies in V_h; GLL quadrature is exact for the products involved,
    # so A u_I = M f exactly (reading C2 must be consistent for this to hold).
    d = dg.Discretisation(2, P, SP2, False, beta, 1.0)
    u = d.nodal(lambda x, y: x * (1 - x) * y * (1 - y))
    f = d.nodal(lambda x, y: 2 * (y * (1 - y) + x * (1 - x)))
    r = d.apply(u) - d.rhs(f)
    assert np.abs(r).max() < 1e-13


@pytest.mark.parametrize("beta", [0.0, 0.5])
def test_dirichlet_polynomial_reproduction_3d(beta):
    d = dg.Discretisation(3, 3, [[0.3, 0.5, 0.2], [0.4, 0.6], [0.5, 0.5]], False, beta, 1.0)
    u = d.nodal(lambda x, y, z: x * (1 - x) * y * (1 - y) * z * (1 - z))
    f = d.nodal(lambda x, y, z: 2 * (y * (1 - y) * z * (1 - z) + x * (1 - x) * z * (1 - z)
                                     + x * (1 - x) * y * (1 - y)))
    assert np.abs(d.apply(u) - d.rhs(f)).max() < 1e-14


def test_3d_reduces_to_2d():
    # reading C1: with z periodic and u constant in z, A_3D u = M_3 (x) A_2D u (L_3 1 = 0)
    sp = [[0.3, 0.5, 0.2], [0.4, 0.35, 0.25], [0.5, 0.5]]
    d3 = dg.Discretisation(3, 3, sp, True, 0.5, 1.0)
    d2 = dg.Discretisation(2, 3, sp[:2], True, 0.5, 1.0)
    rng = np.random.default_rng(0)
    U2 = rng.standard_normal(d2.shape)
    U3 = np.broadcast_to(U2, (d3.shape[0],) + U2.shape).copy()
    V3 = d3.apply(U3)
    V2 = d2.apply(U2)
    ref = d3.axes[2].M[:, None, None] * V2[None]
    assert np.abs(V3 - ref).max() < 1e-13 * np.abs(ref).max()


def test_matrix_free_equals_dense_3d():
    d = dg.Discretisation(3, 2, [[0.3, 0.7], [0.5, 0.5], [0.2, 0.3, 0.5]], False, 0.5, 1.0)
    rng = np.random.default_rng(1)
    U = rng.standard_normal(d.shape)
    assert np.abs(d.apply(U).reshape(-1) - d.dense() @ U.reshape(-1)).max() < 1e-12


def test_spectral_convergence_periodic_2d():
    # Sec. 4 test problem: error of the exact discrete solution decays exponentially in P
    errs = []
    for P in (2, 4, 6, 8):
        d = dg.Discretisation(2, P, [[0.5] * 4, [0.5] * 4], True, 0.0, 1.0)
        f = d.nodal(lambda x, y: 2 * np.pi ** 2 * np.sin(np.pi * x) * np.sin(np.pi * y))
        g = d.rhs(f).reshape(-1)
        A = d.dense()
        u = np.linalg.lstsq(A, g, rcond=1e-10)[0]
        u -= u.mean()
        ue = d.nodal(lambda x, y: np.sin(np.pi * x) * np.sin(np.pi * y)).reshape(-1)
        errs.append(np.abs(u - ue).max())
    assert errs[0] > 1e-2 and errs[-1] < 1e-6
    for a, b in zip(errs, errs[1:]):
        assert b < a / 20


def test_layout_roundtrip():
    rng = np.random.default_rng(2)
    u = rng.standard_normal((2, 3, 4, 5, 5, 5))
    U = to_global(u, 3)
    assert U.shape == (10, 15, 20)
    assert U[5 + 1, 2 * 5 + 3, 3 * 5 + 4] == u[1, 2, 3, 1, 3, 4]
    assert np.array_equal(to_element(U, (4, 3, 2), 5), u)

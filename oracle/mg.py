"""Oracle: p-multigrid V-cycle and inexact multigrid-preconditioned CG (Sec. 3.2-3.3, 4.1).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Levels P_l = 2^l, l = 0..L (Sec. 3.2); A_l is the same discretisation
re-made at order P_l; the prolongation I_l is the embedded interpolation
(coarse Lagrange basis evaluated at the fine GLL nodes), the restriction its
transpose.  Coarse problem: A_0^+ f_0 by conjugate gradients, with the
right-hand side projected onto range(A_0) when A_0 is singular (periodic).

Readings:
  C8  MGCG beta = z^T (r - r_old) / delta (the printed q^T makes the formula
      dimensionally inconsistent); r_old starts at 0, literally as printed.
  C10 Coarse CG runs to a relative residual of 1e-14 (cap 10 N_0 iterations).
  C14 Stop when ||r||_2 <= rtol ||r_0||_2 of the nodal residual g - A u.
"""
from __future__ import annotations

import math

import numpy as np

from .dg import Discretisation, gll, lagrange_eval
from .schwarz import Smoother


def interpolation_1d(Pc: int, Pf: int) -> np.ndarray:
    """J[i, k] = phi_k^{(Pc)}(eta_i^{(Pf)}): embedded interpolation (Sec. 3.2)."""
    eta_c, _ = gll(Pc)
    eta_f, _ = gll(Pf)
    return lagrange_eval(eta_c, eta_f)


class Level:
    def __init__(self, disc: Discretisation, smoother: Smoother | None, ns):
        self.disc = disc
        self.smoother = smoother
        self.ns = ns                           # (pre, post)


class Hierarchy:
    """p-multigrid hierarchy (Sec. 3.2).

    smoother: 'EA' | 'FA' | 'EM' | 'FM'; overlap '0' | 'l'; weighting as in Smoother.
    ns: (pre, post) steps; variable=True -> n_{s,l} = ns * 2^(L-l) (variable V-cycle of
    Sec. 4.3, pinned by the face-centred columns of Table 4).
    coarse: 'cg' (the paper's choice) or 'dense' (pseudo-inverse, tiny grids only).
    """

    def __init__(self, dim, P, spacing, periodic, beta=0.0, mu_star=1.0, smoother="EA",
                 overlap="l", weighting="quintic", ns=(1, 1), variable=False, omega=1.0,
                 coarse="cg", coarse_rtol=1e-14, omega_level=None, tau_level=None):
        """omega_level / tau_level: optional per-level damping and transition width
        (index = level l; entries for l >= 1), overriding omega and tau = 1."""
        L = int(round(math.log2(P)))
        if 2 ** L != P:
            raise ValueError("P must be a power of two (P_l = 2^l)")
        self.dim, self.P, self.L = dim, P, L
        self.periodic = periodic
        self.coarse = coarse
        self.coarse_rtol = coarse_rtol
        self.levels = []
        for l in range(L + 1):
            disc = Discretisation(dim, 2 ** l, spacing, periodic, beta, mu_star)
            sm = None
            nsl = (0, 0)
            if l > 0:
                om = omega_level[l] if omega_level is not None else omega
                ta = tau_level[l] if tau_level is not None else 1.0
                sm = Smoother(disc, smoother, overlap, weighting, om, tau=ta)
                fac = 2 ** (L - l) if variable else 1
                nsl = (ns[0] * fac, ns[1] * fac)
            self.levels.append(Level(disc, sm, nsl))
        self.J = [None] + [interpolation_1d(2 ** (l - 1), 2 ** l) for l in range(1, L + 1)]
        self._dense_pinv = None

    # -- transfers ---------------------------------------------------------
    def prolong(self, l, Uc):
        """I_l u_{l-1}: per element, J along every direction (block diagonal)."""
        disc = self.levels[l].disc
        T = Uc
        for d in range(self.dim):
            ne = disc.axes[d].Ne
            T = disc.along(np.kron(np.eye(ne), self.J[l]), T, d)
        return T

    def restrict(self, l, Rf):
        """I_l^T r_l."""
        disc = self.levels[l].disc
        T = Rf
        for d in range(self.dim):
            ne = disc.axes[d].Ne
            T = disc.along(np.kron(np.eye(ne), self.J[l]).T, T, d)
        return T

    # -- coarse solve --------------------------------------------------------
    def coarse_solve(self, F0):
        disc = self.levels[0].disc
        if self.periodic:
            F0 = F0 - F0.mean()                # projection onto range(A_0) (Kaasschieter)
        if self.coarse == "dense":
            if self._dense_pinv is None:
                # singular values at rounding level (the periodic null space) count as zero
                self._dense_pinv = np.linalg.pinv(disc.dense(), rcond=1e-10, hermitian=True)
            return (self._dense_pinv @ F0.reshape(-1)).reshape(F0.shape)
        return cg(disc.apply, F0, rtol=self.coarse_rtol, maxit=10 * disc.ndof)[0]

    # -- Algorithm 1 ---------------------------------------------------------
    def vcycle(self, U, F):
        L = self.L
        us = [None] * (L + 1)
        fs = [None] * (L + 1)
        us[L], fs[L] = U, F
        for l in range(L, 0, -1):
            lev = self.levels[l]
            if l < L:
                us[l] = np.zeros_like(fs[l])
            us[l] = lev.smoother.smooth(us[l], fs[l], lev.ns[0], post=False)
            fs[l - 1] = self.restrict(l, fs[l] - lev.disc.apply(us[l]))
        us[0] = self.coarse_solve(fs[0])
        for l in range(1, L + 1):
            lev = self.levels[l]
            us[l] = us[l] + self.prolong(l, us[l - 1])
            us[l] = lev.smoother.smooth(us[l], fs[l], lev.ns[1], post=True)
        return us[L]

    @property
    def fine(self):
        return self.levels[self.L].disc


def cg(apply, b, x0=None, rtol=1e-14, maxit=10000):
    """Plain conjugate gradients (Hestenes-Stiefel)."""
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - apply(x)
    p = r.copy()
    rr = float(np.vdot(r, r))
    r0 = math.sqrt(rr)
    if r0 == 0.0:
        return x, 0
    for it in range(1, maxit + 1):
        q = apply(p)
        alpha = rr / float(np.vdot(p, q))
        x = x + alpha * p
        r = r - alpha * q
        rr_new = float(np.vdot(r, r))
        if math.sqrt(rr_new) <= rtol * r0:
            return x, it
        p = r + (rr_new / rr) * p
        rr = rr_new
    return x, maxit


def mgcg(h: Hierarchy, U, F, rtol=1e-10, maxit=100, history=None):
    """Algorithm 2 (inexact PCG, Golub-Ye beta; reading C8).  Returns (u, residual norms)."""
    disc = h.fine
    hist = [] if history is None else history
    r_old = np.zeros_like(F)
    R = F - disc.apply(U)
    r0 = float(np.linalg.norm(R))
    hist.append(r0)
    if r0 == 0.0:
        return U, hist
    Pv = h.vcycle(np.zeros_like(R), R)
    delta = float(np.vdot(Pv, R))
    for _ in range(maxit):
        Q = disc.apply(Pv)
        alpha = delta / float(np.vdot(Pv, Q))
        U = U + alpha * Pv
        R = R - alpha * Q
        rn = float(np.linalg.norm(R))
        hist.append(rn)
        if rn <= rtol * r0:
            break
        Z = h.vcycle(np.zeros_like(R), R)
        beta = float(np.vdot(Z, R - r_old)) / delta
        Pv = Z + beta * Pv
        delta = float(np.vdot(Z, R))
        r_old = R
    return U, hist


def mg(h: Hierarchy, U, F, rtol=1e-10, maxit=100):
    """Stand-alone multigrid: repeated V-cycles on the residual equation (Sec. 3.2)."""
    disc = h.fine
    R = F - disc.apply(U)
    hist = [float(np.linalg.norm(R))]
    for _ in range(maxit):
        U = U + h.vcycle(np.zeros_like(R), R)
        R = F - disc.apply(U)
        hist.append(float(np.linalg.norm(R)))
        if hist[-1] <= rtol * hist[0]:
            break
    return U, hist


def rates(hist, reduction=1e10):
    """rho = (r_n / r_0)^(1/n), rbar = -log10 rho, n10 = cycles to 1e-10 (Eqs. rho, r)."""
    r0 = hist[0]
    n10 = None
    for n, rn in enumerate(hist):
        if n > 0 and rn <= r0 / reduction:
            n10 = n
            break
    n = n10 if n10 is not None else len(hist) - 1
    rho = (hist[n] / r0) ** (1.0 / n)
    return {"rho": rho, "rbar": -math.log10(rho), "n10": n10, "n": n}

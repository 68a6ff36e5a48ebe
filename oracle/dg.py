"""Oracle: nodal IP/LDG discretisation of the Poisson equation (Sec. 2).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The global 1-D stiffness matrix of each axis is assembled row by row from the
element equations in primal form (Eq. "primal form", Sec. 2.4): the volume
term, the lifting terms of the element's two faces and the numerical flux
(Eq. "flux:num:sigma") of those faces.  The d-dimensional operator is the
tensor-product sum of Eq. (discrete problem), Sec. 2.4:

    A = M2 (x) L1 + L2 (x) M1                      (2-D, as printed)
    A = M3 (x) M2 (x) L1 + M3 (x) L2 (x) M1 + L3 (x) M2 (x) M1   (3-D, reading C1)

Readings (the paper is silent or garbled here):
  C2  Homogeneous Dirichlet walls: a ghost element of the same width with the
      odd reflection u_ghost(xi) = -u(-xi), and beta = 0 on wall faces.  This
      is symmetric Nitsche/SIPG with penalty 2 mu at the wall.
  C3  The first terms of L^- and L^+ carry Delta x^m (the element's own width);
      the printed Delta x^{m-1} / Delta x^{m+1} is a typo, the element
      equations give Delta x^m.  Assembling from the element equations (as done
      here) yields this reading automatically.
  C4  The volume term is (2 / Delta x) L^s (Sec. 2.4 element equations).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
from numpy.polynomial import legendre as npleg


# ----------------------------------------------------------------------------
# 1-D spectral building blocks (Sec. 2.4)
# ----------------------------------------------------------------------------

def gll(P: int):
    """GLL nodes eta_0 = -1 < ... < eta_P = 1 and weights rho_i (Sec. 2.4).

    The interior nodes are the roots of L_P'(x) (numpy companion-matrix roots,
    polished by Newton steps on L_P'); rho_i = 2 / (P (P+1) L_P(eta_i)^2).
    """
    if P < 1:
        raise ValueError("P >= 1")
    LP = npleg.Legendre.basis(P)
    dLP = LP.deriv(1)
    d2LP = LP.deriv(2)
    inner = np.sort(np.real(dLP.roots())) if P > 1 else np.zeros(0)
    for _ in range(3):
        if P > 1:
            inner = inner - dLP(inner) / d2LP(inner)
    eta = np.concatenate(([-1.0], inner, [1.0]))
    rho = 2.0 / (P * (P + 1) * LP(eta) ** 2)
    return eta, rho


def lagrange_eval(nodes: np.ndarray, x: np.ndarray) -> np.ndarray:
    """B[i, k] = phi_k(x_i) for the Lagrange polynomials of ``nodes`` (product form)."""
    n = len(nodes)
    B = np.ones((len(x), n))
    for k in range(n):
        for m in range(n):
            if m != k:
                B[:, k] *= (x - nodes[m]) / (nodes[k] - nodes[m])
    return B


def lagrange_deriv(nodes: np.ndarray, x: np.ndarray) -> np.ndarray:
    """B[i, k] = phi_k'(x_i), differentiating the product form term by term."""
    n = len(nodes)
    B = np.zeros((len(x), n))
    for k in range(n):
        for l in range(n):
            if l == k:
                continue
            term = np.full(len(x), 1.0 / (nodes[k] - nodes[l]))
            for m in range(n):
                if m != k and m != l:
                    term = term * (x - nodes[m]) / (nodes[k] - nodes[m])
            B[:, k] += term
    return B


def diff_matrix(eta: np.ndarray) -> np.ndarray:
    """D^s_{ik} = phi_k'(eta_i) (Sec. 2.4)."""
    return lagrange_deriv(eta, eta)


def std_stiffness(rho: np.ndarray, D: np.ndarray) -> np.ndarray:
    """L^s_{ik} = sum_j rho_j D_{ji} D_{jk} (Sec. 2.4, standard 1-D stiffness)."""
    return D.T @ np.diag(rho) @ D


# ----------------------------------------------------------------------------
# Global 1-D operators (Eqs. M:generic, L:generic; assembled from the primal form)
# ----------------------------------------------------------------------------

class Axis1D:
    """Global 1-D mass (diagonal) and stiffness (sparse) matrices of one axis."""

    def __init__(self, P, dx, beta, mu_star, periodic):
        self.P = P
        self.NP = P + 1
        self.dx = np.asarray(dx, dtype=np.float64)
        self.Ne = len(self.dx)
        self.beta = float(beta)
        self.mu_star = float(mu_star)
        self.periodic = bool(periodic)
        self.eta, self.rho = gll(P)
        self.D = diff_matrix(self.eta)
        self.Ls = std_stiffness(self.rho, self.D)
        self.N = self.Ne * self.NP
        self.M = np.concatenate([0.5 * h * self.rho for h in self.dx])
        self.L = self._assemble()
        # physical node coordinates, shape (Ne, NP)
        left = np.concatenate(([0.0], np.cumsum(self.dx)[:-1]))
        self.coords = left[:, None] + 0.5 * (self.eta[None, :] + 1.0) * self.dx[:, None]

    # -- neighbour traces ------------------------------------------------
    def _node(self, m, i):
        """u_i^m as {global column: coefficient}; m may be -1 or Ne (reading C2 for walls)."""
        P, NP, Ne = self.P, self.NP, self.Ne
        if 0 <= m < Ne:
            return {m * NP + i: 1.0}
        if self.periodic:
            return {(m % Ne) * NP + i: 1.0}
        mm = 0 if m < 0 else Ne - 1          # odd reflection of the wall element
        return {mm * NP + (P - i): -1.0}

    def _dx(self, m):
        if 0 <= m < self.Ne:
            return self.dx[m]
        if self.periodic:
            return self.dx[m % self.Ne]
        return self.dx[0] if m < 0 else self.dx[-1]

    def _face_beta(self, left_elem):
        """beta on the face between elements left_elem and left_elem+1 (0 at walls, C2)."""
        if not self.periodic and (left_elem < 0 or left_elem >= self.Ne - 1):
            return 0.0
        return self.beta

    def _deriv(self, m, side):
        """sum_k D^s_{side,k} u_k^m (side = 0 or P) as {column: coefficient}."""
        out = {}
        for k in range(self.NP):
            for c, v in self._node(m, k).items():
                out[c] = out.get(c, 0.0) + self.D[side, k] * v
        return out

    def _penalty(self, a):
        """Bracket of Eq. (flux:num:sigma) on the face between a and a+1: the LDG
        correction terms plus mu = mu0 (1 + mu_star), mu0 the LDG threshold (Sec. 2.4)."""
        b = self._face_beta(a)
        ha, hb = self._dx(a), self._dx(a + 1)
        rP, r0 = self.rho[self.P], self.rho[0]
        mu0 = 1.0 / (2 * ha * rP) + 1.0 / (2 * hb * r0)
        mu = mu0 * (1.0 + self.mu_star)
        return 2 * (b * b + b) / (ha * rP) + 2 * (b * b - b) / (hb * r0) + mu

    def _flux(self, a):
        """Numerical flux sigma_hat on the face between elements a and a+1 (Eq. flux:num:sigma)."""
        b = self._face_beta(a)
        P = self.P
        out = {}

        def add(d, s):
            for c, v in d.items():
                out[c] = out.get(c, 0.0) + s * v
        add(self._deriv(a, P), (1 + 2 * b) / self._dx(a))
        add(self._deriv(a + 1, 0), (1 - 2 * b) / self._dx(a + 1))
        c = self._penalty(a)
        add(self._node(a + 1, 0), c)
        add(self._node(a, P), -c)
        return out

    def _assemble(self):
        P, NP, Ne = self.P, self.NP, self.Ne
        rows, cols, vals = [], [], []

        def add(row, d, s):
            for c, v in d.items():
                rows.append(row)
                cols.append(c)
                vals.append(s * v)

        for m in range(Ne):
            h = self.dx[m]
            bl = self._face_beta(m - 1)
            br = self._face_beta(m)
            jump_l = {}
            for c, v in self._node(m, 0).items():
                jump_l[c] = jump_l.get(c, 0.0) + v
            for c, v in self._node(m - 1, P).items():
                jump_l[c] = jump_l.get(c, 0.0) - v
            jump_r = {}
            for c, v in self._node(m + 1, 0).items():
                jump_r[c] = jump_r.get(c, 0.0) + v
            for c, v in self._node(m, P).items():
                jump_r[c] = jump_r.get(c, 0.0) - v
            flux_l = self._flux(m - 1)
            flux_r = self._flux(m)
            for i in range(NP):
                row = m * NP + i
                # volume term (2 / dx) L^s u^m (C4)
                for k in range(NP):
                    rows.append(row)
                    cols.append(m * NP + k)
                    vals.append(2.0 / h * self.Ls[i, k])
                # lifting of the face jumps (terms 2 and 3 of the element equations)
                add(row, jump_l, (1 - 2 * bl) / h * self.D[0, i])
                add(row, jump_r, (1 + 2 * br) / h * self.D[P, i])
                # boundary flux terms: + delta_{i0} sigma_hat(m-1/2) - delta_{iP} sigma_hat(m+1/2)
                if i == 0:
                    add(row, flux_l, 1.0)
                if i == P:
                    add(row, flux_r, -1.0)
        L = sp.coo_matrix((vals, (rows, cols)), shape=(self.N, self.N)).tocsr()
        L.sum_duplicates()
        return L

    def dense_L(self):
        return self.L.toarray()


# ----------------------------------------------------------------------------
# d-dimensional operator (Eq. discrete problem; 3-D by reading C1)
# ----------------------------------------------------------------------------

class Discretisation:
    """Nodal DG operator on a Cartesian grid; vectors in the global layout U[Z][Y][X]."""

    def __init__(self, dim, P, spacing, periodic, beta=0.0, mu_star=1.0):
        self.dim = dim
        self.P = P
        self.NP = P + 1
        self.periodic = periodic
        self.beta = beta
        self.mu_star = mu_star
        self.spacing = [np.asarray(s, dtype=np.float64) for s in spacing]
        self.axes = [Axis1D(P, self.spacing[d], beta, mu_star, periodic) for d in range(dim)]
        self.n_elem = tuple(a.Ne for a in self.axes)
        self.shape = tuple(a.N for a in reversed(self.axes))    # (Z, Y, X)
        self.ndof = int(np.prod(self.shape))

    def axis_of(self, d):
        """numpy axis of spatial direction d (x is the last axis)."""
        return self.dim - 1 - d

    def along(self, mat, U, d):
        """Apply a 1-D matrix (dense, sparse or a diagonal given as 1-D array) along direction d."""
        ax = self.axis_of(d)
        if isinstance(mat, np.ndarray) and mat.ndim == 1:
            sh = [1] * self.dim
            sh[ax] = -1
            return U * mat.reshape(sh)
        V = np.moveaxis(U, ax, 0)
        s = V.shape
        W = mat @ V.reshape(s[0], -1)
        return np.moveaxis(np.asarray(W).reshape((mat.shape[0],) + s[1:]), 0, ax)

    def apply(self, U):
        """A U = sum_d (M ... L_d ... M) U."""
        V = np.zeros_like(U)
        for d in range(self.dim):
            T = U
            for e in range(self.dim):
                T = self.along(self.axes[e].L if e == d else self.axes[e].M, T, e)
            V += T
        return V

    def mass(self, U):
        for e in range(self.dim):
            U = self.along(self.axes[e].M, U, e)
        return U

    def rhs(self, F):
        """g = M f (Sec. 2.4: g_ij = (dx1 dx2 / 4) rho_i rho_j f(x_ij))."""
        return self.mass(F)

    def dense(self):
        """Dense A (only for tiny grids): kron(M3, M2, L1) + ... with x fastest."""
        mats = []
        for d in range(self.dim):
            factors = []
            for e in range(self.dim):
                factors.append(self.axes[e].dense_L() if e == d else np.diag(self.axes[e].M))
            K = factors[self.dim - 1]
            for e in range(self.dim - 2, -1, -1):
                K = np.kron(K, factors[e])
            mats.append(K)
        return sum(mats)

    def coords(self):
        return [a.coords for a in self.axes]

    def nodal(self, fn):
        """Evaluate fn at the nodes (global layout)."""
        xs = [np.concatenate(a.coords) for a in self.axes]
        grids = np.meshgrid(*reversed(xs), indexing="ij")    # Z, Y, X order
        return fn(*reversed(grids))

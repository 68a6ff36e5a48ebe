"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds no arithmetic of the solver method.  It only describes the
problems (grid sizes, element widths, boundary type, flux parameter) and draws
seeded random numbers with NumPy's PCG64 generator.  Node coordinates are NOT
computed here: each side (oracle, CUDA library) evaluates the analytic
right-hand sides at its own Gauss-Lobatto-Legendre nodes.

Workloads follow the shapes used in Stiller, "Robust multigrid for high-order
DG" (arXiv 1603.02524): the 2-D periodic Lottes-Fischer test of Sec. 4
(u = sin(pi x) sin(pi y) on (0, 2AR) x (0, 2)) and its 3-D homogeneous
Dirichlet analogue on the unit cube.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Workload:
    """A problem description: grid, boundary type and discretisation knobs."""

    name: str
    dim: int
    P: int
    n_elem: tuple                       # elements per axis (x, y[, z])
    spacing: list                       # per axis: list of element widths
    periodic: bool                      # True: periodic, False: homogeneous Dirichlet
    beta: float = 0.0                   # LDG auxiliary parameter (0 => IP), Sec. 2.3
    mu_star: float = 1.0                # penalty factor, Sec. 2.4 (mu = mu0 (1 + mu_star))
    rhs: str = "sin"                    # "sin" | "noise" | "sin+noise" | "gauss"
    seed: int = 0
    notes: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def ndof(self) -> int:
        return int(np.prod(self.n_elem)) * (self.P + 1) ** self.dim

    def lengths(self):
        return [float(np.sum(s)) for s in self.spacing]


def uniform_spacing(n: int, length: float) -> list:
    return [length / n] * n


def geometric_spacing(n: int, h0: float, ratio_total: float) -> list:
    """Widths h0 * q**k, k = 0..n-1, with q = ratio_total**(1/(n-1))."""
    if n == 1:
        return [h0]
    q = ratio_total ** (1.0 / (n - 1))
    return [h0 * q ** k for k in range(n)]


def config1() -> Workload:
    """2-D unit square, 4x4 elements, P=4, IP, Dirichlet, f = 2 pi^2 sin sin."""
    return Workload("poisson2d_4x4_P4_dirichlet", 2, 4, (4, 4),
                    [uniform_spacing(4, 1.0)] * 2, periodic=False, rhs="sin")


def config2(beta: float = 0.0) -> Workload:
    """3-D unit cube, 16^3 elements, P=8 (2 985 984 DOF), f = 3 pi^2 sin sin sin + U[-1,1]."""
    return Workload("poisson3d_16cube_P8_dirichlet" + ("_ldg" if beta else "_ip"), 3, 8,
                    (16, 16, 16), [uniform_spacing(16, 1.0)] * 3, periodic=False,
                    beta=beta, rhs="sin+noise")


def config3() -> Workload:
    """3-D unit cube, 32^3 elements, P=16 (160 989 184 DOF)."""
    return Workload("poisson3d_32cube_P16_dirichlet_ip", 3, 16, (32, 32, 32),
                    [uniform_spacing(32, 1.0)] * 3, periodic=False, rhs="sin+noise")


def config4() -> Workload:
    """3-D stretched grid 64x16x8, P=8; widths h q^k with aspect ratios 1..32."""
    h = 1.0 / 64
    sx = uniform_spacing(64, 1.0)
    sy = geometric_spacing(16, h, 32.0)
    sz = geometric_spacing(8, h, 32.0)
    return Workload("poisson3d_64x16x8_P8_stretched", 3, 8, (64, 16, 8), [sx, sy, sz],
                    periodic=False, rhs="gauss")


def paper_periodic_2d(n: int, P: int, aspect: int = 1, beta: float = 0.0) -> Workload:
    """Sec. 4 test: (0, 2AR) x (0, 2), n x n elements, periodic, f = 2 pi^2 sin sin."""
    return Workload(f"paper2d_{n}x{n}_P{P}_AR{aspect}", 2, P, (n, n),
                    [uniform_spacing(n, 2.0 * aspect), uniform_spacing(n, 2.0)],
                    periodic=True, beta=beta, rhs="sin")


def small_3d(n=(3, 3, 3), P=4, periodic=False, beta=0.0, spacing=None) -> Workload:
    sp = spacing or [uniform_spacing(k, 1.0) for k in n]
    return Workload(f"small3d_{'x'.join(map(str, n))}_P{P}", 3, P, tuple(n), sp,
                    periodic=periodic, beta=beta, rhs="noise")


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def element_shape(w: Workload, P: int | None = None) -> tuple:
    """Element-major array shape: (n_z, n_y, n_x, N_P, N_P, N_P) in 3-D, (n_y, n_x, N_P, N_P) in 2-D."""
    NP = (w.P if P is None else P) + 1
    ne = tuple(reversed(w.n_elem))
    return ne + (NP,) * w.dim


def uniform_noise(w: Workload, seed: int | None = None, P: int | None = None) -> np.ndarray:
    """U[-1, 1] nodal values in the element-major layout (fp64)."""
    g = rng(w.seed if seed is None else seed)
    return g.uniform(-1.0, 1.0, size=element_shape(w, P))


def gauss_noise(w: Workload, seed: int | None = None, P: int | None = None) -> np.ndarray:
    g = rng(w.seed if seed is None else seed)
    return g.standard_normal(size=element_shape(w, P))


def unit_uniform(w: Workload, seed: int | None = None, P: int | None = None) -> np.ndarray:
    """U[0, 1] values (the random initial guess of Sec. 4)."""
    g = rng(w.seed if seed is None else seed)
    return g.uniform(0.0, 1.0, size=element_shape(w, P))


def sin_source(dim: int):
    """f = dim pi^2 prod sin(pi x_d): -lap of u = prod sin(pi x_d)."""
    c = dim * math.pi ** 2

    def f(*xs):
        out = c
        for x in xs:
            out = out * np.sin(math.pi * x)
        return out
    return f


def sin_solution(dim: int):
    def u(*xs):
        out = 1.0
        for x in xs:
            out = out * np.sin(math.pi * x)
        return out
    return u


def nodal_field(w: Workload, fn, coords_1d: list) -> np.ndarray:
    """Evaluate fn at the nodes, given per-axis nodal coordinates.

    ``coords_1d[d]`` has shape (n_elem[d], N_P): the physical coordinate of node i
    of element m along axis d, as computed by the caller's own discretisation.
    The result uses the element-major layout.
    """
    if w.dim == 2:
        X = coords_1d[0][None, :, None, :]
        Y = coords_1d[1][:, None, :, None]
        return fn(X, Y) * np.ones(element_shape(w))
    X = coords_1d[0][None, None, :, None, None, :]
    Y = coords_1d[1][None, :, None, None, :, None]
    Z = coords_1d[2][:, None, None, :, None, None]
    return fn(X, Y, Z) * np.ones(element_shape(w))


def source_values(w: Workload, coords_1d: list) -> np.ndarray:
    """Nodal source f for the workload (before multiplication by the mass matrix)."""
    if w.rhs == "sin":
        return nodal_field(w, sin_source(w.dim), coords_1d)
    if w.rhs == "sin+noise":
        return nodal_field(w, sin_source(w.dim), coords_1d) + uniform_noise(w)
    if w.rhs == "noise":
        return uniform_noise(w)
    if w.rhs == "gauss":
        return gauss_noise(w)
    raise ValueError(w.rhs)


BATCH_SIDES = (8, 12, 16, 24)      # elements per axis of a batched grid
BATCH_ORDERS = (4, 8, 16, 32)


def config5(n_grids: int = 64, n_rhs: int = 4, budget_dof: int = 512_000_000,
            grid_cap_dof: int = 80_000_000, seed: int = 0) -> list:
    """Batched solves: n_grids independent 3-D Dirichlet grids on (0,1) x (0,ry) x (0,rz)
    with n^3 elements, n drawn from BATCH_SIDES and P from BATCH_ORDERS; widths
    hx = 1/n, hy = ry/n, hz = rz/n with ry, rz log-uniform in [1/4, 4], so element
    aspect ratios span 1..16; n_rhs seeded Gaussian right-hand sides per grid.  The
    device-memory budget caps the draws: a draw whose DOF x n_rhs exceeds grid_cap_dof,
    or the remaining budget less what the grids still to draw need at the smallest
    size, is rejected and redrawn; each accepted grid records its draw number in
    `notes`."""
    g = rng(seed)
    out, left, draws = [], int(budget_dof), 0
    smallest = min(BATCH_SIDES) ** 3 * (min(BATCH_ORDERS) + 1) ** 3 * n_rhs
    while len(out) < n_grids:
        draws += 1
        if draws > 1000 * n_grids:
            raise RuntimeError("batch budget too small for the requested number of grids")
        n = int(g.choice(BATCH_SIDES))
        P = int(g.choice(BATCH_ORDERS))
        ry, rz = (float(v) for v in np.exp(g.uniform(math.log(0.25), math.log(4.0), size=2)))
        dof = n ** 3 * (P + 1) ** 3
        if dof * n_rhs > min(grid_cap_dof, left - (n_grids - len(out) - 1) * smallest):
            continue
        left -= dof * n_rhs
        k = len(out)
        out.append(Workload(f"batch{k:02d}_{n}cube_P{P}", 3, P, (n, n, n),
                            [uniform_spacing(n, 1.0), uniform_spacing(n, ry), uniform_spacing(n, rz)],
                            periodic=False, rhs="gauss", seed=seed * 100003 + k, notes=f"draw {draws}",
                            extra={"n_rhs": n_rhs, "aspect": (1.0, ry, rz)}))
    return out

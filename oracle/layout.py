"""Element-major <-> global tensor layout (test infrastructure only).

Element-major layout (the CUDA library's layout): ``u[e_z][e_y][e_x][k][j][i]``
with x fastest inside an element.  Global layout (the oracle's working layout):
``U[Z][Y][X]`` with the global 1-D index ``X = e_x * N_P + i`` of Eq. (IJ),
Sec. 2.4.
"""
import numpy as np


def to_global(u: np.ndarray, dim: int) -> np.ndarray:
    if dim == 2:
        ny, nx, NP, _ = u.shape
        return u.transpose(0, 2, 1, 3).reshape(ny * NP, nx * NP)
    nz, ny, nx, NP, _, _ = u.shape
    return u.transpose(0, 3, 1, 4, 2, 5).reshape(nz * NP, ny * NP, nx * NP)


def to_element(U: np.ndarray, n_elem, NP: int) -> np.ndarray:
    dim = U.ndim
    if dim == 2:
        nx, ny = n_elem[0], n_elem[1]
        return np.ascontiguousarray(U.reshape(ny, NP, nx, NP).transpose(0, 2, 1, 3))
    nx, ny, nz = n_elem
    return np.ascontiguousarray(U.reshape(nz, NP, ny, NP, nx, NP).transpose(0, 2, 4, 1, 3, 5))

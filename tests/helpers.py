"""Shared helpers of the parity tests: matching oracle / CUDA-library objects."""
import numpy as np

from oracle.layout import to_element, to_global


def to_dev(a, dev="cuda"):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a).reshape(-1)).to(dev)


def from_dev(t, shape):
    return t.detach().cpu().numpy().reshape(shape)


def elem_shape(dim, n_elem, P):
    NP = P + 1
    return tuple(reversed(n_elem[:dim])) + (NP,) * dim


def g2e(U, n_elem, P):
    return to_element(U, n_elem, P + 1)


def e2g(u, dim):
    return to_global(u, dim)


def rel_err(got, ref):
    scale = np.abs(ref).max()
    return np.abs(got - ref).max() / (scale if scale > 0 else 1.0)

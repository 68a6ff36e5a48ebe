"""GB300-native p-multigrid solver for nodal IP/LDG discretisations of the Poisson
equation on Cartesian grids (Stiller, arXiv 1603.02524).

The solver is the C-ABI library ``_build/libpmg.so`` (CUDA, sm_103a); this package
holds its sources (``csrc/``), the build script and a thin ctypes binding.
Nothing here falls back to a CPU implementation: without the built library every
call raises.
"""
from .binding import Batch, Grid, Hierarchy, PmgError, load  # noqa: F401

__all__ = ["Grid", "Hierarchy", "PmgError", "load", "build"]


def build(verbose: bool = False) -> str:
    from .build import build as _build
    return _build(verbose=verbose)

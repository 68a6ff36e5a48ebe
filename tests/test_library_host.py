"""CPU-side checks of the C-ABI library: it loads, exports every declared symbol,
and its host-only entry points (argument checks, node coordinates) behave."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1603_02524_gb300.build import build
    build()
    from paper_1603_02524_gb300 import binding
    return binding.load()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "pmg.h")).read()
    return sorted(set(re.findall(r"^(?:int|void|const char\*)\s+(pmg_\w+)\(", src, re.M)))


def test_header_declares_entry_points():
    names = declared_functions()
    for n in ("pmg_grid_create", "pmg_hierarchy_build", "pmg_apply", "pmg_rhs", "pmg_smooth",
              "pmg_solve", "pmg_restrict", "pmg_prolong", "pmg_coarse_solve", "pmg_vcycle"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for n in declared_functions():
        assert hasattr(lib, n), n


def test_status_strings(lib):
    assert lib.pmg_status_string(0) == b"ok"
    assert b"invalid" in lib.pmg_status_string(-1)


def test_grid_argument_checks(lib):
    from paper_1603_02524_gb300 import Grid, PmgError
    sp = [[0.5, 0.5]] * 3
    with pytest.raises(PmgError):
        Grid(3, 3, (2, 2, 2), sp, periodic=False)        # P not a power of two
    with pytest.raises(PmgError):
        Grid(3, 64, (2, 2, 2), sp, periodic=False)       # P <= 32
    with pytest.raises(PmgError):
        Grid(4, 2, (2, 2, 2), sp, periodic=False)
    with pytest.raises(PmgError):
        Grid(2, 2, (1, 2), [[1.0], [0.5, 0.5]], periodic=True)   # periodic needs >= 2 elements
    with pytest.raises(PmgError):
        Grid(2, 2, (2, 2), [[0.5, -0.5], [0.5, 0.5]], periodic=False)
    Grid(2, 32, (2, 2), [[0.5, 0.5]] * 2, periodic=True).close()
    Grid(3, 32, (2, 2, 2), sp, periodic=False).close()


def test_node_coordinates_match_oracle(lib):
    from oracle import dg
    from paper_1603_02524_gb300 import Grid
    sp = [[0.3, 0.5, 0.2], [0.25, 0.75], [1.0]]
    for P in (1, 2, 4, 8, 16):
        g = Grid(3, P, (3, 2, 1), sp, periodic=False)
        for d in range(3):
            ref = dg.Axis1D(P, sp[d], 0.0, 1.0, False).coords
            assert np.abs(g.coords(d) - ref).max() < 1e-15
        g.close()

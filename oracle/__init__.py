"""Plain, slow FP64 CPU oracle of the p-multigrid DG Poisson solver.

Stiller, "Robust multigrid for high-order discontinuous Galerkin methods: a
fast Poisson solver suitable for high-aspect ratio Cartesian grids"
(arXiv 1603.02524).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import this package.  The
CUDA library never uses it and shares no code with it: it has its own GLL
nodes, operator blocks, eigen-solver and patch tables.

Modules
-------
dg       -- GLL nodes, 1-D matrices, the nodal IP/LDG operator (Sec. 2), RHS.
schwarz  -- element- and face-centred subdomains, weights, fast diagonalisation,
            additive (EA, FA) and multiplicative (EM, FM) Schwarz (Sec. 3.1).
mg       -- p-levels, embedded interpolation, V-cycle (Algorithm 1), coarse CG,
            inexact PCG (Algorithm 2), convergence metrics (Sec. 4.1).
layout   -- element-major <-> global tensor layout conversion.

Every function names the passage of the paper it follows.  Readings of
passages that are garbled, ambiguous or silent are labelled C1..C18 in the
docstrings; "parity unpinned" marks a function no test pins to something
outside the oracle (the 3-D convergence *rates*, for which the paper has no
numbers, are the only such case).
"""

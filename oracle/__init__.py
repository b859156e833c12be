"""FP64 CPU oracle of the complex additive multilevel cycle.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU legs of ``bench.py``; never by the product package.
"""
from .helmholtz import (  # noqa: F401
    ADD, HB, DLINEAR, HIERARCHICAL,
    JACOBI, UCG, LGRID, EXP, TRANSITION,
    Hierarchy, Level, axis_spacing, cells_per_axis, cpoint_mask,
    element_matrices, element_matrices_1d, fmg_start, helmholtz_element,
    inject, omega_scheme, prolong, restrict, rotated_cells, zero_boundary,
)

"""Seeded synthetic inputs (magnetic field cubes and seed lists) shared by the
oracle tests, the CUDA parity tests and the benchmark.

This package only *generates inputs*: it samples analytic or point-source
magnetic fields on uniform or stretched (rectilinear) grids. It holds none of the method's arithmetic
(no curl, no interpolation, no tracing, no Q), so both the CPU oracle and the
CUDA library can be fed from it without sharing any computation.
"""
from .fields import (  # noqa: F401
    Grid,
    RectGrid,
    stretched_axis,
    stretched_grid,
    monopole24_stretched,
    analytic_cube,
    monopole_cube,
    random_charges,
    quadrupole_charges,
    quadrupole_cube,
    twist_tube_cube,
    perturbed_charges,
    random_smooth_cube,
    batch_specs,
    ANALYTIC_GRID,
    monopole24_cube,
    large_monopole,
    adjoint_cubes,
)

"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package holds no arithmetic of the discontinuous Galerkin method: only
meshes (vertex coordinates and element-to-vertex lists), initial-condition and
bed functions of the physical coordinates, parameter presets for the dam-break
workloads, and seeded random fields.  Whoever consumes these inputs evaluates
the functions at its own node coordinates.
"""
from .meshes import interval_mesh, rect_tri_mesh  # noqa: F401
from .cases import (  # noqa: F401
    Case, dam_break_1d, radial_dam_2d, bump_dam_2d, slump_2d, lake_at_rest_1d, dry_dam_2d,
    parallel_surface_1d, paper_dam_break_1d, random_smooth_fields, ensemble_cases,
    REG_NONE, REG_SMOOTH_MAX, REG_LOCAL_QUAD, REG_TANH, REG_EXP, REG_BIVISC,
    BC_COPY, BC_DIRICHLET, BC_WALL,
)

"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package describes inputs only: mesh topology, vertex and curved
geometry-node coordinates, material fields, initial data, source and receiver
positions, and the tabulated fewer-point volume rules (quadrature.py: stored
points and weights, an input like the paper's tabulated rules).  It holds none
of the discretisation arithmetic (no basis, no geometric factors, no
operators, no rule construction at run time); the oracle and the CUDA library
each compute those on their own from what is produced here.
"""
from .warped_cube import (  # noqa: F401
    CONFIGS,
    lattice_tet,
    lattice_tri,
    kuhn_cube,
    warp_displacement,
    geometry_nodes,
    warped_cube,
    standing_wave,
    OMEGA,
    c2_heterogeneous,
    c2_perturbed_samples,
    ricker,
    source_positions,
    receiver_positions,
    random_fields,
)
from .quadrature import SYMMETRIC_RULES, symmetric_rule, fewer_point_rule  # noqa: F401

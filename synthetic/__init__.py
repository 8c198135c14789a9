"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package describes inputs only: mesh topology, vertex and curved
geometry-node coordinates, material fields, initial data, source and receiver
positions.  It holds none of the discretisation arithmetic (no quadrature, no
basis, no geometric factors, no operators); the oracle and the CUDA library
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

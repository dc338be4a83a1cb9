"""Seeded synthetic inputs for the SIBFA water workloads.

This package only draws numbers: water geometries, per-molecule multipoles,
velocities and the force-field parameter table.  It holds none of the
method's arithmetic (no energies, potentials or forces), so both the FP64
oracle and the CUDA path may read what it produces.
"""
from .water import (  # noqa: F401
    PARAMS,
    WATER_GEOM,
    N_SITES,
    N_LP,
    System,
    make_box,
    make_cluster,
    make_cluster_batch,
    make_cluster_sizes,
    make_dimer,
    make_ortho_box,
    make_config,
    maxwell_velocities,
    random_rotation,
    general_multipoles,
    with_general_multipoles,
)
